"""Parity on the largest grids: 2D at N = 1024, the largest N the library accepts and the
finest grid of the paper's 2D studies (fine grid 2048^2, three-halves grid 1536^2), and 3D
at N = 256 (fine grid 512^3, 1.6 GB per FP32 field), the largest 3D grid.

These sizes take the general transform paths (line lengths 384 to 2048 have no warp-level
plan, and the longest lines leave room for only one or two lines per block). Transforms are
compared on sampled modes and points, which the oracle evaluates one by one; the 2D
Navier-Stokes sub-steps are compared in full. Point sets mix uniform points (including
coordinates outside [0, L)) with a dense closed curve or surface, so that both sparse and
crowded bins occur.

Tolerances: 1e-10 relative in FP64 mode, 1e-5 in mixed mode (2-norm; 10x that against the
largest entry), as for the smaller parity cases.
"""
import numpy as np
import pytest

from oracle import spectral as sp
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
NTOL = {"fp64": 1e-12, "mixed": 1e-6}
CDT = {"fp64": np.complex128, "mixed": np.complex64}


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


def sample_modes(rng, N, d, n):
    """Random modes of the half spectrum (m_x >= 0, no Nyquist index) plus corner modes.
    Returns the array index (slowest axis first) and the integer modes (m_x, m_y[, m_z])."""
    h = N // 2
    ix = rng.integers(0, h, n)
    iy = rng.integers(0, N, n)
    iz = rng.integers(0, N, n)
    iy[iy == h] = 0
    iz[iz == h] = 0
    corners = [(0, 0, 0), (h - 1, 0, 0), (0, h - 1, 0), (0, 0, h - 1), (h - 1, h + 1, h + 1),
               (1, N - 1, N - 1), (h - 1, h - 1, h - 1)]
    ix = np.concatenate([ix, [q[0] for q in corners]])
    iy = np.concatenate([iy, [q[1] for q in corners]])
    iz = np.concatenate([iz, [q[2] for q in corners]])
    m = sp.mode_ints(N)
    if d == 2:
        return (iy, ix), np.stack([ix, m[iy]], axis=1)
    return (iz, iy, ix), np.stack([ix, m[iy], m[iz]], axis=1)


def sample_points(rng, M, n):
    return np.unique(np.concatenate([rng.integers(0, M, n), [0, M // 2 - 1, M // 2, M - 1]]))


def test_grids_beyond_the_largest_transform_are_rejected(lib, torch_mod):
    with pytest.raises(lib.FsibError) as ei:
        lib.Problem(1026, 2, 10, 1.0, 1.0, 1e-3, 1e-6)   # N above the accepted range
    assert ei.value.code == -1
    with pytest.raises(lib.FsibError) as ei:
        lib.Problem(258, 3, 10, 1.0, 1.0, 1e-3, 1e-6)    # 3D fine grid 576 > 512
    assert ei.value.code == -6


# --- 2D, N = 1024 -----------------------------------------------------------------------------

N2, M2 = 1024, 6000


@pytest.fixture(scope="module")
def case2d():
    rng = np.random.default_rng(10240)
    Xu = rng.uniform(-0.5, 1.5, (2, M2 // 2))
    Xc = wl.ellipse(M2 - M2 // 2, 0.3, 0.3, (0.5, 0.5))
    X = np.ascontiguousarray(np.concatenate([Xu, Xc], axis=1))
    c = rng.standard_normal((2, M2))
    H = half_random(rng, 2, N2)
    return X, c, H


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_2d_largest_grid_spread_sampled_modes_and_interp_sampled_points(lib, torch_mod, case2d, prec):
    torch = torch_mod
    X, c, H = case2d
    pb = lib.Problem(N2, 2, M2, 1.0, 0.0, 1e-3, NTOL[prec], precision=prec)
    fh = pb.spread(cuda(X, torch), cuda(c, torch))
    Hc = H.astype(CDT[prec])          # the library sees the spectrum in its transform type
    U = pb.interp(cuda(Hc, torch), cuda(X, torch))
    torch.cuda.synchronize()
    rng = np.random.default_rng(10241)
    (iy, ix), modes = sample_modes(rng, N2, 2, 400)
    got = to_np(fh)[:, iy, ix].astype(np.complex128)
    ref = sp.spread_at_modes(X, c, modes)
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]
    idx = sample_points(rng, M2, 150)
    Uref = sp.interp_direct(sp.half_to_full(Hc.astype(np.complex128), N2, 2), X[:, idx], N2)
    Ug = to_np(U)[:, idx]
    assert rel2(Ug, Uref) <= TOL[prec]
    assert relmax(Ug, Uref) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_2d_largest_grid_ns_substeps(lib, torch_mod, prec):
    """Both Navier-Stokes sub-steps with the three-halves products on the 1536^2 grid."""
    torch = torch_mod
    rng = np.random.default_rng(10242)
    mu, rho, dt = 0.05, 1.3, 0.002
    cd = CDT[prec]
    u0 = sp.leray(sp.half_to_full(half_random(rng, 2, N2), N2, 2), N2)
    f = sp.half_to_full(half_random(rng, 2, N2), N2, 2)
    f_in = sp.half_to_full(sp.full_to_half(f, N2).astype(cd).astype(np.complex128), N2, 2)
    u_in = sp.half_to_full(sp.full_to_half(u0, N2).astype(cd).astype(np.complex128), N2, 2)
    pb = lib.Problem(N2, 2, 4, mu, rho, dt, NTOL[prec], precision=prec)
    ft = cuda(sp.full_to_half(f, N2).astype(cd), torch)
    ut = cuda(sp.full_to_half(u0, N2).astype(cd), torch)
    uh = pb.new_spec()
    pb.fluid_step(ft, ut, uh)
    torch.cuda.synchronize()
    rh, r1 = sp.ns_substeps(f_in, u_in, N2, mu, rho, dt)
    gh = sp.half_to_full(to_np(uh).astype(np.complex128), N2, 2)
    g1 = sp.half_to_full(to_np(ut).astype(np.complex128), N2, 2)
    assert rel2(gh, rh) <= TOL[prec]
    assert rel2(g1, r1) <= TOL[prec]
    assert sp.max_divergence(g1, N2) <= (1e-6 if prec == "mixed" else 1e-13)


# --- 3D, N = 256 ------------------------------------------------------------------------------

N3, M3 = 256, 30000


@pytest.fixture(scope="module")
def case3d():
    rng = np.random.default_rng(2560)
    Xu = rng.uniform(-0.25, 1.25, (3, M3 // 2))
    Xs, _ = wl.icosphere(5, 0.25, (0.5, 0.5, 0.5))   # 10242 vertices on a sphere
    X = np.ascontiguousarray(np.concatenate([Xu, Xs], axis=1))
    M = X.shape[1]
    c = rng.standard_normal((3, M))
    H = half_random(rng, 3, N3, 1e-2)
    return X, c, H


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_3d_N256_spread_sampled_modes_and_interp_sampled_points(lib, torch_mod, case3d, prec):
    torch = torch_mod
    X, c, H = case3d
    M = X.shape[1]
    pb = lib.Problem(N3, 3, M, 1.0, 0.0, 1e-3, NTOL[prec], precision=prec)
    fh = pb.spread(cuda(X, torch), cuda(c, torch))
    Hc = H.astype(CDT[prec])
    U = pb.interp(cuda(Hc, torch), cuda(X, torch))
    torch.cuda.synchronize()
    rng = np.random.default_rng(2561)
    (iz, iy, ix), modes = sample_modes(rng, N3, 3, 193)
    got = to_np(fh)[:, iz, iy, ix].astype(np.complex128)
    ref = sp.spread_at_modes(X, c, modes)
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]
    idx = sample_points(rng, M, 60)
    Uref = sp.interp_direct(sp.half_to_full(Hc.astype(np.complex128), N3, 3), X[:, idx], N3)
    Ug = to_np(U)[:, idx]
    assert rel2(Ug, Uref) <= TOL[prec]
    assert relmax(Ug, Uref) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_3d_N256_ns_step_of_a_shear_flow(lib, torch_mod, prec):
    """A property that holds at any size: u = (sin 2 pi y + cos 4 pi z, 0, 0) is divergence-free
    and its nonlinear term vanishes (u_x does not depend on x), so with no force each mode
    of the Navier-Stokes step (Algorithm 1) is only damped: u^{m+1/2} = u^m / (1 + a) and
    u^{m+1} = u^m (1 - a) / (1 + a), a = mu dt |k|^2 / (2 rho). On the 384^3 dealiasing grid
    this runs the block-level product pass with the longest lines of a 3D plan."""
    torch = torch_mod
    N, mu, rho, dt = N3, 0.05, 1.0, 0.01
    F = np.zeros((3, N, N, N), dtype=np.complex128)     # [c][z][y][x], FFT order
    F[0, 0, 1, 0], F[0, 0, N - 1, 0] = -0.5j, 0.5j      # sin(2 pi y)
    F[0, 2, 0, 0], F[0, N - 2, 0, 0] = 0.5, 0.5         # cos(4 pi z)
    m = sp.mode_ints(N).astype(np.float64)
    k2 = (2 * np.pi) ** 2 * (m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    a = mu * dt * k2 / (2 * rho)
    half_ref = F / (1 + a)[None]
    one_ref = F * ((1 - a) / (1 + a))[None]
    cd = CDT[prec]
    pb = lib.Problem(N, 3, 4, mu, rho, dt, NTOL[prec], precision=prec)
    ft = cuda(np.zeros_like(sp.full_to_half(F, N)).astype(cd), torch)
    ut = cuda(sp.full_to_half(F, N).astype(cd), torch)
    uh = pb.new_spec()
    pb.fluid_step(ft, ut, uh)
    torch.cuda.synchronize()
    assert rel2(sp.half_to_full(to_np(uh).astype(np.complex128), N, 3), half_ref) <= TOL[prec]
    assert rel2(sp.half_to_full(to_np(ut).astype(np.complex128), N, 3), one_ref) <= TOL[prec]
