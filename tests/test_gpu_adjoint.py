"""GPU reverse mode of the quasi-static Stokes stepper against the oracle's adjoint and FP64
finite differences."""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import spectral as sp
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-9, "mixed": 1e-4}


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def case3d():
    Xref, tri = wl.latlong_sphere(5, 10, 0.25, (0.5, 0.48, 0.52))
    X0 = 0.5 + (Xref - 0.5) * np.array([[1.12], [0.92], [1.04]])
    return Xref, tri, X0


def make(lib, N, d, M, prec, dt=2e-3):
    return lib.Problem(N, d, M, 1.0, 0.0, dt, 1e-12 if prec == "fp64" else 1e-6, precision=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_interp_grad_matches_oracle(lib, torch_mod, prec):
    torch = torch_mod
    rng = np.random.default_rng(3)
    N, M = 12, 200
    X = rng.uniform(-0.2, 1.2, (3, M))
    H = rng.standard_normal((3, N, N, N // 2)) + 1j * rng.standard_normal((3, N, N, N // 2))
    pb = make(lib, N, 3, M, prec)
    Ht = torch.from_numpy(H.astype(np.complex128 if prec == "fp64" else np.complex64)).cuda()
    G = pb.interp_grad(Ht, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = ad.grad_at_points(sp.half_to_full(H, N, 3), X, N)
    assert rel2(G, ref) <= (1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rollout_adjoint_matches_oracle(lib, torch_mod, prec):
    torch = torch_mod
    Xref, tri, X0 = case3d()
    N, K, ck, dt, sigma = 10, 5, 2, 2e-3, 1.0
    M = X0.shape[1]
    pb = make(lib, N, 3, M, prec, dt)
    pb.set_force_mesh(tri, Xref, sigma)
    center, R = np.array([0.5, 0.48, 0.52]), 0.25
    force = st.mesh_model(Xref, tri, sigma)
    g_ref, s_ref, XK = ad.rollout_grad(X0, K, force, sigma, N, 1.0, dt, lambda X: ad.sphere_loss(X, center, R)[1])
    dL = torch.from_numpy(ad.sphere_loss(XK, center, R)[1]).cuda()
    g0, gs = pb.step_adjoint(torch.from_numpy(X0).cuda(), K, ck, dL)
    assert rel2(g0.cpu().numpy(), g_ref) <= TOL[prec]
    assert abs(float(gs.cpu()) - s_ref) <= TOL[prec] * abs(s_ref)


def test_autograd_function_matches_finite_differences(lib, torch_mod):
    torch = torch_mod
    Xref, tri, X0 = case3d()
    N, K, ck, dt = 10, 4, 3, 2e-3
    M = X0.shape[1]
    pb = make(lib, N, 3, M, "fp64", dt)
    center = torch.tensor([0.5, 0.48, 0.52], dtype=torch.float64, device="cuda")[:, None]

    def loss(X0t, sig):
        XK = lib.stokes_rollout(X0t, sig, pb, K, ck, tri, Xref)
        r = torch.sqrt(((XK - center) ** 2).sum(0))
        return ((r - 0.25) ** 2).sum()

    X0t = torch.from_numpy(X0.copy()).cuda().requires_grad_(True)
    sig = torch.tensor(1.1, dtype=torch.float64, requires_grad=True)
    L = loss(X0t, sig)
    L.backward()
    rng = np.random.default_rng(5)
    with torch.no_grad():
        for _ in range(2):
            v = torch.from_numpy(rng.standard_normal(X0.shape)).cuda()
            eps = 1e-6
            fd = (loss(X0t + eps * v, sig) - loss(X0t - eps * v, sig)) / (2 * eps)
            an = (X0t.grad * v).sum()
            assert abs(float(fd - an)) <= 1e-6 * abs(float(fd))
        e = 1e-6
        fds = (loss(X0t, sig + e) - loss(X0t, sig - e)) / (2 * e)
        assert abs(float(fds) - float(sig.grad)) <= 1e-6 * abs(float(fds))
