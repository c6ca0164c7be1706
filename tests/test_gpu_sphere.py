"""Parity of the three-dimensional sphere problems (Secs. 6.2.3, 6.2.4) with the oracle.

Refined-icosahedron spheres of radius L/3 in the sine flow u_0 = (sin 2 pi z, 0, sin 2 pi y),
with cot-weight springs (elastic) or surface tension, through the C ABI: FP64 mode to 1e-10
relative, FP32-mixed to 1e-5; the last cases run the paper's N = 32, four refinements
(M = 2562) configuration.
"""
import numpy as np
import pytest

from oracle import lagrangian as lg
from oracle import spectral as sp
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
NTOL = {"fp64": 1e-12, "mixed": 1e-6}
CDT = {"fp64": np.complex128, "mixed": np.complex64}


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_np(t):
    return t.detach().cpu().numpy()


def cuda(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("level", [1, 3, 4])
def test_tension_force_and_energy_match_oracle(lib, torch_mod, level):
    torch = torch_mod
    X, tri = wl.icosphere(level, 0.3, (0.5, 0.45, 0.6))
    rng = np.random.default_rng(level)
    X = X + rng.uniform(-0.01, 0.01, X.shape)
    M = X.shape[1]
    pb = lib.Problem(16, 3, M, 0.01, 1.0, 1e-3, 1e-12)
    pb.set_force_tension(tri, 1.3)
    c = to_np(pb.force(cuda(X, torch)))
    ref = lg.surface_tension_force(X, tri, 1.3)
    assert rel2(c, ref) <= 1e-13
    inv = pb.invariants(cuda(X, torch))
    assert inv["Ep"] == pytest.approx(1.3 * lg.surface_area(X, tri), rel=1e-13)
    assert inv["volume"] == pytest.approx(lg.enclosed_volume(X, tri), rel=1e-13)
    pb.set_force_tension(cuda(tri, torch), 0.5)      # device copy of the triangles
    assert rel2(to_np(pb.force(cuda(X, torch))), ref * (0.5 / 1.3)) <= 1e-13


def test_tension_rejects_bad_meshes(lib, torch_mod):
    pb = lib.Problem(16, 3, 4, 0.01, 1.0, 1e-3, 1e-12)
    with pytest.raises(lib.FsibError):
        pb.set_force_tension(np.array([[0, 1, 4]], dtype=np.int32), 1.0)
    with pytest.raises(lib.FsibError):
        pb.set_force_tension(np.array([[0, 1, 1]], dtype=np.int32), 1.0)
    p2 = lib.Problem(16, 2, 4, 0.01, 1.0, 1e-3, 1e-12)
    with pytest.raises(lib.FsibError):
        p2.set_force_tension(np.array([[0, 1, 2]], dtype=np.int32), 1.0)


def _run(lib, torch, prob, prec, nsteps):
    pb = lib.Problem(prob.N, 3, prob.M, prob.mu, prob.rho, prob.dt, NTOL[prec], precision=prec)
    if prob.force == "mesh":
        pb.set_force_mesh(prob.tri, prob.Xref, prob.stiffness)
        force = st.mesh_model(prob.Xref, prob.tri, prob.stiffness)
    else:
        pb.set_force_tension(prob.tri, prob.stiffness)
        force = st.tension_model(prob.tri, prob.stiffness)
    Xt = cuda(prob.X0, torch)
    ut = cuda(prob.extra["u0"].astype(CDT[prec]), torch)
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=nsteps)
    inv = pb.invariants(Xt, ut)
    torch.cuda.synchronize()
    N = prob.N
    X, u = prob.X0.copy(), sp.half_to_full(prob.extra["u0"], N, 3)
    U = sp.interp_direct(u, X, N)
    for _ in range(nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt)
    tol = TOL[prec]
    assert rel2(to_np(Xt) - prob.X0, X - prob.X0) <= tol * (10 if prec == "mixed" else 1)
    assert rel2(sp.half_to_full(to_np(ut).astype(np.complex128), N, 3), u) <= tol
    assert rel2(to_np(Ut), U) <= tol
    assert inv["volume"] == pytest.approx(lg.enclosed_volume(to_np(Xt), prob.tri), rel=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", ["elastic", "tension"])
def test_sphere_steps_match_oracle(lib, torch_mod, model, prec):
    """Two refinements (M = 162), N = 12, four steps of dt = 2e-3."""
    prob = wl.config_ns3d_sphere(model, level=2, N=12, dt=2e-3, precision=prec)
    _run(lib, torch_mod, prob, prec, 4)


@pytest.mark.parametrize("model", ["elastic", "tension"])
def test_sphere_paper_configuration_matches_oracle(lib, torch_mod, model):
    """The paper's N = 32, four refinements (M = 2562), dt = 1e-3: two FP64 steps."""
    prob = wl.config_ns3d_sphere(model)
    _run(lib, torch_mod, prob, "fp64", 2)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model", ["elastic", "tension"])
def test_sphere_coarsest_grid_matches_oracle(lib, torch_mod, model, prec):
    """The convergence study's first level: N = 4 (the smallest plan: N/2 = 2 modes along x,
    a 6^3 dealiasing grid), one refinement (M = 42), dt = 0.004."""
    prob = wl.config_ns3d_sphere(model, level=1, N=4, dt=0.004, precision=prec)
    _run(lib, torch_mod, prob, prec, 5)
