"""Parity at the benchmark sizes, in the launch configuration the benchmark times.

The workloads are the benchmark's (3D Navier-Stokes N = 64, M = 10082, FP64; N = 128,
M = 40322, FP32-mixed; the differentiable 3D Stokes problem N = 96, M = 20002, mixed),
with the launch shapes chosen by the autotuner as in bench.py. Large transforms are
checked on sampled outputs that the oracle computes one by one (type-1 modes, type-2
points); the fluid update and one whole FP64 step are checked in full.

Tolerances: 1e-10 relative in FP64 mode, 1e-5 relative in mixed mode (2-norm over the
sample; 10x that against the largest sampled entry).
"""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
NUFFT_TOL = {"fp64": 1e-12, "mixed": 1e-6}   # the tolerances the benchmark plans with
CDT = {"fp64": np.complex128, "mixed": np.complex64}

CONFIGS = {
    "ns3d_N64_fp64": (wl.config_ns3d_fp64, "fp64"),
    "ns3d_N128_mixed": (wl.config_ns3d_mixed, "mixed"),
    "stokes3d_N96_mixed": (wl.config_stokes3d_adjoint, "mixed"),
}


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def to_np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def cuda(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def half_random(rng, d, N, scale=1.0):
    shape = (d,) + (N,) * (d - 1) + (N // 2,)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def setup(lib, torch, name, u0=None):
    """The benchmark's problem object for one workload, with autotuned launch shapes."""
    make_prob, prec = CONFIGS[name]
    prob = make_prob()
    pb = lib.Problem(prob.N, prob.d, prob.M, prob.mu, prob.rho, prob.dt, NUFFT_TOL[prec], precision=prec)
    pb.set_force_mesh(prob.tri, cuda(prob.Xref, torch), prob.stiffness)
    X = cuda(prob.X0, torch)
    if prob.rho > 0:
        u = cuda(u0.astype(CDT[prec]), torch) if u0 is not None else pb.new_spec()
        U = pb.interp(u, X)
        pb.autotune(X, u, U)
    else:
        pb.autotune(X)
    return prob, prec, pb


def sample_modes(rng, N, n):
    """Random integer modes of the half spectrum (m_x >= 0, no Nyquist index), plus corners."""
    h = N // 2
    ix = rng.integers(0, h, n)
    iy = rng.integers(0, N, n)
    iz = rng.integers(0, N, n)
    iy[iy == h] = 0
    iz[iz == h] = 0
    corners = [(0, 0, 0), (h - 1, 0, 0), (0, h - 1, 0), (0, 0, h - 1), (h - 1, h + 1, h + 1),
               (1, N - 1, N - 1), (h - 1, h - 1, h - 1)]
    ix = np.concatenate([ix, [c[0] for c in corners]])
    iy = np.concatenate([iy, [c[1] for c in corners]])
    iz = np.concatenate([iz, [c[2] for c in corners]])
    m = sp.mode_ints(N)
    modes = np.stack([ix, m[iy], m[iz]], axis=1)   # (n, 3) as (m_x, m_y, m_z)
    return (iz, iy, ix), modes


@pytest.mark.parametrize("name", list(CONFIGS))
def test_fullsize_spread_sampled_modes(lib, torch_mod, name):
    torch = torch_mod
    prob, prec, pb = setup(lib, torch, name)
    X0 = prob.X0
    c = st.mesh_model(prob.Xref, prob.tri, prob.stiffness)(X0)   # oracle force, FP64
    fh = pb.spread(cuda(X0, torch), cuda(c, torch))
    torch.cuda.synchronize()
    got_half = to_np(fh).astype(np.complex128)
    rng = np.random.default_rng(7001)
    (iz, iy, ix), modes = sample_modes(rng, prob.N, 249)
    got = got_half[:, iz, iy, ix]
    ref = sp.spread_at_modes(X0, c, modes)
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("name", list(CONFIGS))
def test_fullsize_interp_sampled_points(lib, torch_mod, name):
    torch = torch_mod
    prob, prec, pb = setup(lib, torch, name)
    N = prob.N
    rng = np.random.default_rng(7002)
    uh = half_random(rng, 3, N, 1e-2)
    U = pb.interp(cuda(uh.astype(CDT[prec]), torch), cuda(prob.X0, torch))
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([rng.integers(0, prob.M, 60), [0, 1, prob.M - 1, prob.M // 2]]))
    full = sp.half_to_full(uh.astype(CDT[prec]).astype(np.complex128), N, 3)
    ref = sp.interp_direct(full, prob.X0[:, idx], N)
    got = to_np(U)[:, idx]
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("name", ["ns3d_N64_fp64", "ns3d_N128_mixed"])
def test_fullsize_ns_substeps(lib, torch_mod, name):
    torch = torch_mod
    make_prob, prec = CONFIGS[name]
    prob = make_prob()
    N = prob.N
    rng = np.random.default_rng(7003)
    u0 = sp.leray(sp.half_to_full(half_random(rng, 3, N, 0.05), N, 3), N)
    f = sp.half_to_full(half_random(rng, 3, N, 10.0), N, 3)
    _, _, pb = setup(lib, torch, name, u0=sp.full_to_half(u0, N))
    cd = CDT[prec]
    # the oracle takes the inputs as the library sees them (rounded to the transform type)
    f_in = sp.half_to_full(sp.full_to_half(f, N).astype(cd).astype(np.complex128), N, 3)
    u_in = sp.half_to_full(sp.full_to_half(u0, N).astype(cd).astype(np.complex128), N, 3)
    ft = cuda(sp.full_to_half(f, N).astype(cd), torch)
    ut = cuda(sp.full_to_half(u0, N).astype(cd), torch)
    uh = pb.new_spec()
    pb.fluid_step(ft, ut, uh)
    torch.cuda.synchronize()
    rh, r1 = sp.ns_substeps(f_in, u_in, N, prob.mu, prob.rho, prob.dt)
    gh = sp.half_to_full(to_np(uh).astype(np.complex128), N, 3)
    g1 = sp.half_to_full(to_np(ut).astype(np.complex128), N, 3)
    assert rel2(gh, rh) <= TOL[prec]
    assert rel2(g1, r1) <= TOL[prec]
    assert sp.max_divergence(g1, N) <= (1e-6 if prec == "mixed" else 1e-13)


def test_fullsize_ns_step_fp64(lib, torch_mod):
    """One whole step of the FP64 headline workload (N = 64, M = 10082) against the oracle."""
    torch = torch_mod
    prob = wl.config_ns3d_fp64()
    N = prob.N
    rng = np.random.default_rng(7004)
    u0 = sp.leray(sp.half_to_full(half_random(rng, 3, N, 0.02), N, 3), N)
    _, _, pb = setup(lib, torch, "ns3d_N64_fp64", u0=sp.full_to_half(u0, N))
    Xt = cuda(prob.X0, torch)
    ut = cuda(sp.full_to_half(u0, N), torch)
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=1)
    torch.cuda.synchronize()
    force = st.mesh_model(prob.Xref, prob.tri, prob.stiffness)
    X0 = prob.X0
    U0 = sp.interp_direct(u0, X0, N)
    X1, u1, U1 = st.ns_step(X0.copy(), u0.copy(), U0, force, N, prob.mu, prob.rho, prob.dt)
    assert rel2(to_np(Xt) - X0, X1 - X0) <= TOL["fp64"]
    assert rel2(sp.half_to_full(to_np(ut), N, 3), u1) <= TOL["fp64"]
    assert rel2(to_np(Ut), U1) <= TOL["fp64"]


def test_fullsize_mixed_steps_keep_invariants(lib, torch_mod):
    """Ten mixed steps of the N = 128 workload: divergence-free and zero-mean velocity."""
    torch = torch_mod
    prob, prec, pb = setup(lib, torch, "ns3d_N128_mixed")
    X = cuda(prob.X0, torch)
    u = pb.new_spec()
    U = pb.interp(u, X)
    pb.step(X, u, U, nsteps=10)
    torch.cuda.synchronize()
    Xn = to_np(X)
    assert np.all(np.isfinite(Xn))
    full = sp.half_to_full(to_np(u).astype(np.complex128), prob.N, 3)
    assert np.max(np.abs(full)) > 0
    assert sp.max_divergence(full, prob.N) <= 1e-6
    assert np.max(np.abs(full[:, 0, 0, 0])) <= 1e-5 * np.max(np.abs(full))
