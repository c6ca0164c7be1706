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
