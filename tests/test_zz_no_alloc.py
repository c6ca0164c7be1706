"""The allocation-free type-1 spread (fsib_spread_static) against the handle-based one.

Callers that cannot allocate device memory (a host framework whose allocator
owns the GPU, or loops that cannot afford cudaMalloc's implicit device
synchronisation) use fsib_spread_static, whose scratch is a fixed static device
array. This file is collected last on purpose. Each case makes two calls in a
row on different inputs, so stale contents left in the shared scratch by the
first call would show up in the second.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
NTOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_08694_gb300 import build as fbuild
    from paper_2302_08694_gb300 import fsib
    fbuild.build()
    return torch, fsib


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d,N,M", [(3, 16, 900), (2, 32, 300), (3, 24, 37)])
def test_static_spread_matches_handle_spread_twice(env, prec, d, N, M):
    torch, fsib = env
    lib = fsib.load()
    pb = fsib.Problem(N, d, M, 1.0, 1.0, 1e-3, NTOL[prec], precision=prec)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    for call in range(2):
        rng = np.random.default_rng(1000 * call + 7 * d + N + M)
        X = torch.from_numpy(rng.uniform(-0.4, 1.6, (d, M))).cuda()
        F = torch.from_numpy(rng.standard_normal((d, M))).cuda()
        om = torch.from_numpy(rng.uniform(0.5, 1.5, M)).cuda() if call == 1 else None
        ref = pb.spread(X, F, om).cpu().numpy()
        out = torch.full(pb.spec_shape, float("nan"), dtype=cdt, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.fsib_spread_static(N, d, M, NTOL[prec], 0 if prec == "fp64" else 1,
                                    X.data_ptr(), F.data_ptr(), om.data_ptr() if om is not None else None,
                                    out.data_ptr(), stream)
        assert rc == 0, lib.fsib_static_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel2(got, ref) <= TOL[prec]


def test_static_spread_rejects_oversized_problem(env):
    torch, fsib = env
    lib = fsib.load()
    X = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.complex128, device="cuda")
    rc = lib.fsib_spread_static(256, 3, 8, 1e-12, 0, X.data_ptr(), X.data_ptr(), None, out.data_ptr(), None)
    assert rc == -1
    assert "static scratch" in lib.fsib_static_last_error().decode()


def _static(lib, N, d, M, prec, X, F, out, stream=None):
    return lib.fsib_spread_static(N, d, M, NTOL[prec], 0 if prec == "fp64" else 1, X.data_ptr(), F.data_ptr(),
                                  None, out.data_ptr(), stream)


def test_static_spread_at_the_scratch_limit(env):
    """The largest 3D FP64 problem at N = 48 that fits the 64 MiB scratch is accepted and matches
    fsib_spread; one more point is rejected. The boundary is found by bisection on M: a rejected
    call enqueues nothing and reports the bytes it needed."""
    torch, fsib = env
    lib = fsib.load()
    d, N, prec = 3, 48, "fp64"
    Mhi = 2_000_000
    rng = np.random.default_rng(4848)
    X = torch.from_numpy(rng.uniform(0.0, 1.0, (d, Mhi))).cuda()
    F = torch.from_numpy(rng.standard_normal((d, Mhi))).cuda()
    out = torch.zeros((d, N, N, N // 2), dtype=torch.complex128, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def rejected(M):
        rc = _static(lib, N, d, M, prec, X[:, :M].contiguous(), F[:, :M].contiguous(), out, stream)
        if rc == 0:
            return False
        assert rc == -1 and "static scratch" in lib.fsib_static_last_error().decode()
        return True

    assert rejected(Mhi)
    lo, hi = 1, Mhi           # lo accepted, hi rejected
    assert not rejected(lo)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if rejected(mid):
            hi = mid
        else:
            lo = mid
    assert lo > 100_000       # the cap is reached through the points, not the grids
    torch.cuda.synchronize()
    Xm, Fm = X[:, :lo].contiguous(), F[:, :lo].contiguous()
    pb = fsib.Problem(N, d, lo, 1.0, 1.0, 1e-3, NTOL[prec], precision=prec)
    ref = pb.spread(Xm, Fm).cpu().numpy()
    out.fill_(float("nan"))
    assert _static(lib, N, d, lo, prec, Xm, Fm, out, stream) == 0, lib.fsib_static_last_error().decode()
    torch.cuda.synchronize()
    assert rel2(out.cpu().numpy(), ref) <= TOL[prec]
    assert _static(lib, N, d, lo + 1, prec, X[:, :lo + 1].contiguous(), F[:, :lo + 1].contiguous(), out,
                   stream) == -1
    assert "static scratch" in lib.fsib_static_last_error().decode()


def test_static_spread_replays_in_a_cuda_graph(env):
    """After one call with the same sizes outside capture (which uploads the tables), the call
    enqueues only kernels and memsets, so it can be captured in a CUDA graph; the graph,
    replayed twice on new inputs copied into the captured buffers, matches fsib_spread. Under
    capture, a call whose tables are not in the scratch is refused without enqueueing anything."""
    torch, fsib = env
    lib = fsib.load()
    d, N, M, prec = 3, 16, 700, "mixed"
    pb = fsib.Problem(N, d, M, 1.0, 1.0, 1e-3, NTOL[prec], precision=prec)
    X = torch.empty((d, M), dtype=torch.float64, device="cuda")
    F = torch.empty_like(X)
    out = torch.zeros(pb.spec_shape, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    rng = np.random.default_rng(99)
    X.copy_(torch.from_numpy(rng.uniform(0.0, 1.0, (d, M))))
    F.copy_(torch.from_numpy(rng.standard_normal((d, M))))
    torch.cuda.synchronize()
    assert _static(lib, N, d, M, prec, X, F, out, ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        rc = _static(lib, N, d, M, prec, X, F, out, ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, lib.fsib_static_last_error().decode()
    for rep in range(2):
        X.copy_(torch.from_numpy(rng.uniform(-0.5, 1.5, (d, M))))
        F.copy_(torch.from_numpy(rng.standard_normal((d, M))))
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref = pb.spread(X, F).cpu().numpy()
        assert rel2(out.cpu().numpy(), ref) <= TOL[prec]
    # other sizes under capture: refused, nothing enqueued
    g2 = torch.cuda.CUDAGraph()
    out2 = torch.zeros((d, 20, 20, 10), dtype=torch.complex64, device="cuda")
    with torch.cuda.graph(g2, stream=s, capture_error_mode="thread_local"):
        rc2 = lib.fsib_spread_static(20, d, M, 1e-6, 1, X.data_ptr(), F.data_ptr(), None, out2.data_ptr(),
                                     ctypes.c_void_p(s.cuda_stream))
        msg = lib.fsib_static_last_error().decode()
        out2.zero_()
    assert rc2 == -1 and "outside stream capture" in msg
