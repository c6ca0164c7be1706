"""Parity of the two-dimensional validation problems (Secs. 5.2.1, 5.2.2) with the oracle.

The target-point spring force, the uniform body force in the Navier-Stokes update and
the channel flux diagnostic, through the C ABI, against the FP64 oracle: FP64 mode to
1e-10 relative, FP32-mixed mode to 1e-5 (the fluxes are sums in double of the stored
coefficients and match to 1e-12 in both modes).
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


def problem(lib, prob, prec, N=None):
    N = N or prob.N
    return lib.Problem(N, prob.d, prob.M, prob.mu, prob.rho, prob.dt, NTOL[prec], precision=prec)


@pytest.mark.parametrize("d", [2, 3])
def test_target_force_and_energy_match_oracle(lib, torch_mod, d):
    torch = torch_mod
    rng = np.random.default_rng(40 + d)
    M, K, omega = 37, 2.5e3, 0.0625
    X = rng.uniform(0, 1, (d, M))
    Xt = X + rng.uniform(-0.02, 0.02, (d, M))
    pb = lib.Problem(16, d, M, 0.1, 1.0, 1e-3, 1e-12)
    pb.set_force_target(Xt, K, omega)            # host copy of the targets
    c = to_np(pb.force(cuda(X, torch)))
    ref = st.target_model(Xt, K, omega)(X)
    assert rel2(c, ref) <= 1e-14
    inv = pb.invariants(cuda(X, torch))
    assert inv["volume"] == 0.0
    assert inv["Ep"] == pytest.approx(lg.target_energy(X, Xt, K, omega), rel=1e-13)
    pb.set_force_target(cuda(Xt, torch), 2 * K, omega)   # device copy, new stiffness
    assert rel2(to_np(pb.force(cuda(X, torch))), 2 * ref) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d,N,comp,axis", [(2, 8, 0, 1), (2, 16, 1, 0), (2, 24, 0, 0), (3, 8, 0, 1),
                                           (3, 12, 2, 2), (3, 12, 1, 0)])
def test_band_flux_matches_oracle(lib, torch_mod, prec, d, N, comp, axis):
    torch = torch_mod
    rng = np.random.default_rng(1000 + 7 * N + axis)
    H = wl.random_half_spectrum(rng, d, N).astype(CDT[prec])
    pb = lib.Problem(N, d, 5, 0.1, 1.0, 1e-3, NTOL[prec], precision=prec)
    full = sp.half_to_full(H.astype(np.complex128), N, d)
    for y0, y1 in [(0.25, 0.75), (0.13, 0.4), (0.9, 0.35)]:
        got = pb.band_flux(cuda(H, torch), comp, axis, y0, y1)
        want = sp.band_flux(full, N, comp, axis, y0, y1)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-13 * np.max(np.abs(H)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [8, 16])
def test_poiseuille_steps_match_oracle(lib, torch_mod, prec, N):
    """Channel walls on target springs, body force f0 = 100, from rest (reduced run)."""
    torch = torch_mod
    prob = wl.config_poiseuille(N=N)
    ex = prob.extra
    nsteps = 12
    rng = np.random.default_rng(N)
    X0 = prob.X0 + rng.uniform(-0.2, 0.2, prob.X0.shape) / N   # markers off their targets
    pb = problem(lib, prob, prec)
    pb.set_force_target(ex["Xtarget"], prob.stiffness, ex["omega"])
    pb.set_body_force(ex["fbody"])
    Xt = cuda(X0, torch)
    ut = pb.new_spec()
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=nsteps)
    torch.cuda.synchronize()
    force = st.target_model(ex["Xtarget"], prob.stiffness, ex["omega"])
    X, u = X0.copy(), np.zeros((2, N, N), dtype=np.complex128)
    U = np.zeros_like(X)
    for _ in range(nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt, fbody=ex["fbody"])
    tol = TOL[prec]
    assert rel2(to_np(Xt) - X0, X - X0) <= tol * (10 if prec == "mixed" else 1)
    g = sp.half_to_full(to_np(ut).astype(np.complex128), N, 2)
    assert rel2(g, u) <= tol
    assert rel2(to_np(Ut), U) <= tol
    y0, y1 = ex["band"]
    assert pb.band_flux(ut, 0, 1, y0, y1) == pytest.approx(sp.band_flux(u, N, 0, 1, y0, y1), rel=tol)


def test_body_force_change_reaches_the_captured_step(lib, torch_mod):
    """A body force set after a step graph was captured applies to the next step."""
    torch = torch_mod
    prob = wl.config_poiseuille(N=8)
    ex = prob.extra
    pb = problem(lib, prob, "fp64")
    pb.set_force_target(ex["Xtarget"], prob.stiffness, ex["omega"])
    Xt = cuda(prob.X0, torch)
    ut = pb.new_spec()
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=2)            # no body force: nothing moves
    torch.cuda.synchronize()
    assert np.max(np.abs(to_np(ut))) == 0.0
    pb.set_body_force(ex["fbody"])
    pb.step(Xt, ut, Ut, nsteps=1)
    pb.set_body_force((0.0, 0.0))
    pb.step(Xt, ut, Ut, nsteps=1)
    torch.cuda.synchronize()
    force = st.target_model(ex["Xtarget"], prob.stiffness, ex["omega"])
    X, u, U = prob.X0.copy(), np.zeros((2, 8, 8), dtype=np.complex128), np.zeros((2, 16))
    X, u, U = st.ns_step(X, u, U, force, 8, prob.mu, prob.rho, prob.dt, fbody=ex["fbody"])
    X, u, U = st.ns_step(X, u, U, force, 8, prob.mu, prob.rho, prob.dt)
    assert rel2(sp.half_to_full(to_np(ut), 8, 2), u) <= TOL["fp64"]
    assert rel2(to_np(Xt) - prob.X0, X - prob.X0) <= TOL["fp64"]


def test_body_force_needs_navier_stokes(lib, torch_mod):
    pb = lib.Problem(16, 2, 8, 1.0, 0.0, 1e-3, 1e-12)
    with pytest.raises(lib.FsibError) as e:
        pb.set_body_force((1.0, 0.0))
    assert e.value.code == -6
    pb.set_force_target(np.zeros((2, 8)), 1.0, 0.1)
    with pytest.raises(lib.FsibError) as e:
        pb.step_adjoint(np.zeros((2, 8)), 2, 1, np.zeros((2, 8)))
    assert e.value.code == -6
    with pytest.raises(lib.FsibError):
        pb.set_force_target(np.zeros((2, 8)), 1.0, 0.0)


@pytest.mark.parametrize("prec,N,Nb,nsteps", [("fp64", 16, 50, 6), ("mixed", 16, 50, 6), ("fp64", 64, 202, 3)])
def test_sine_circle_steps_match_oracle(lib, torch_mod, prec, N, Nb, nsteps):
    """Circle of radius L/4 released in u_0 = (0, sin 2 pi x) (Sec. 5.2.1); the last case
    is the paper's N = 64, N_b = 202, dt = 1e-3 configuration."""
    torch = torch_mod
    prob = wl.config_ns2d_circle(N=N, Nb=Nb, precision=prec)
    pb = problem(lib, prob, prec)
    pb.set_force_curve(prob.stiffness)
    Xt = cuda(prob.X0, torch)
    ut = cuda(prob.extra["u0"].astype(CDT[prec]), torch)
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=nsteps)
    inv = pb.invariants(Xt, ut)
    torch.cuda.synchronize()
    force = st.curve_model(prob.stiffness)
    X, u = prob.X0.copy(), sp.half_to_full(prob.extra["u0"], N, 2)
    U = sp.interp_direct(u, X, N)
    for _ in range(nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt)
    tol = TOL[prec]
    assert rel2(to_np(Xt) - prob.X0, X - prob.X0) <= tol * (10 if prec == "mixed" else 1)
    assert rel2(sp.half_to_full(to_np(ut).astype(np.complex128), N, 2), u) <= tol
    assert rel2(to_np(Ut), U) <= tol
    assert inv["volume"] == pytest.approx(lg.enclosed_area(to_np(Xt)), rel=1e-12)
