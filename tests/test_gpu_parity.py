"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Tolerances: FP64 mode must match the oracle to 1e-10 relative (2-norm and
element-wise against the largest entry); FP32-mixed mode to 1e-5 relative.
Sizes span several bins and FFT tiles with ragged tails; points include
coordinates outside [0, L) (the library wraps them periodically).
"""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle import stepper as st
from oracle import lagrangian as lg
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp64native": 1e-10, "mixed": 1e-5}
NTOL = {"fp64": 1e-12, "fp64native": 1e-12, "mixed": 1e-6}
CDT = {"fp64": np.complex128, "fp64native": np.complex128, "mixed": np.complex64}


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def to_np(t):
    return t.detach().cpu().numpy()


def cuda(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def half_random(rng, d, N):
    shape = (d,) + (N,) * (d - 1) + (N // 2,)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make(lib, N, d, M, prec, mu=1.0, rho=0.0, dt=1e-3, **kw):
    """fp64: double-float transforms (default FP64 mode); fp64native: FP64 arithmetic."""
    pb = lib.Problem(N, d, M, mu, rho, dt, NTOL[prec], precision="mixed" if prec == "mixed" else "fp64", **kw)
    if prec == "fp64native":
        pb.set_option("native_fp64", 1)
    return pb


# --- type-1 / type-2 against the direct sums --------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp64native", "mixed"])
@pytest.mark.parametrize("d,N,M", [(2, 16, 300), (2, 24, 37), (3, 8, 50), (3, 16, 700), (3, 12, 1),
                                   (3, 36, 150), (3, 72, 211)])
def test_spread_matches_oracle(lib, torch_mod, prec, d, N, M):
    torch = torch_mod
    rng = np.random.default_rng(100 + d * N + M)
    X = rng.uniform(-0.7, 1.9, (d, M))
    F = rng.standard_normal((d, M))
    om = rng.uniform(0.5, 1.5, M)
    pb = make(lib, N, d, M, prec)
    fh = pb.spread(cuda(X, torch), cuda(F, torch), cuda(om, torch))
    torch.cuda.synchronize()
    ref = sp.full_to_half(sp.spread_direct(X, F * om[None, :], N), N)
    got = to_np(fh)
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spread_dense_points_many_slices(lib, torch_mod, prec):
    """Uniform points dense enough that a gather box would need more than 16 slices of 128
    candidates: the slices grow instead, and split boxes are summed from their partials."""
    torch = torch_mod
    rng = np.random.default_rng(321)
    d, N, M = 3, 16, 20000
    X = rng.uniform(0.0, 1.0, (d, M))
    F = rng.standard_normal((d, M))
    pb = make(lib, N, d, M, prec)
    pb.set_option("spread_slice", 128)
    for _ in range(2):  # twice: the work counters and partial counts start from zero each call
        fh = pb.spread(cuda(X, torch), cuda(F, torch))
        torch.cuda.synchronize()
        ref = sp.full_to_half(sp.spread_direct(X, F, N), N)
        got = to_np(fh)
        assert rel2(got, ref) <= TOL[prec]
        assert relmax(got, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spread_dense_curve_2d_shared_boxes(lib, torch_mod, prec):
    """A dense closed curve in 2D (about 300 points per fine cell along it): several blocks share
    each box's candidates and the last one adds their partial boxes in slice order."""
    torch = torch_mod
    rng = np.random.default_rng(654)
    d, N, M = 2, 32, 20000
    th = np.sort(rng.uniform(0.0, 2 * np.pi, M))
    X = np.stack([0.5 + 0.2 * np.cos(th), 0.45 + 0.15 * np.sin(th)])
    F = rng.standard_normal((d, M))
    pb = make(lib, N, d, M, prec)
    ref = sp.full_to_half(sp.spread_direct(X, F, N), N)
    for _ in range(2):  # twice: the per-box counters return to zero
        fh = pb.spread(cuda(X, torch), cuda(F, torch))
        torch.cuda.synchronize()
        got = to_np(fh)
        assert rel2(got, ref) <= TOL[prec]
        assert relmax(got, ref) <= 10 * TOL[prec]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("d,N,M", [(2, 32, 3000), (3, 16, 20000), (3, 24, 997)])
def test_mixed_spread_summation_modes(lib, torch_mod, mode, d, N, M):
    """The FP32 gather spread's three summations (plain FMAs, compensated per term, compensated
    per staged chunk of candidates) all match the direct sums at the mixed tolerance, on dense
    point sets whose cells collect hundreds of terms, and split 3D boxes into several slices."""
    torch = torch_mod
    rng = np.random.default_rng(500 + 7 * mode + d * N + M)
    X = rng.uniform(0.3, 0.6, (d, M))          # clustered: many terms per cell
    F = rng.standard_normal((d, M))
    pb = make(lib, N, d, M, "mixed")
    pb.set_option("spread_sum", mode)
    assert pb.info("spread_sum") == mode
    fh = pb.spread(cuda(X, torch), cuda(F, torch))
    torch.cuda.synchronize()
    ref = sp.full_to_half(sp.spread_direct(X, F, N), N)
    got = to_np(fh)
    assert rel2(got, ref) <= TOL["mixed"]
    assert relmax(got, ref) <= 10 * TOL["mixed"]


def test_spread_sum_option_is_checked(lib, torch_mod):
    pb = make(lib, 8, 3, 10, "mixed")
    assert pb.info("spread_sum") == 2              # compensated per chunk of candidates by default
    with pytest.raises(lib.FsibError):
        pb.set_option("spread_sum", 3)


@pytest.mark.parametrize("prec", ["fp64", "fp64native", "mixed"])
@pytest.mark.parametrize("d,N,M", [(2, 16, 300), (2, 24, 37), (3, 8, 50), (3, 16, 700), (3, 12, 1),
                                   (3, 72, 211)])
def test_interp_matches_oracle(lib, torch_mod, prec, d, N, M):
    torch = torch_mod
    rng = np.random.default_rng(200 + d * N + M)
    X = rng.uniform(-0.5, 1.5, (d, M))
    H = half_random(rng, d, N)
    pb = make(lib, N, d, M, prec)
    Ht = cuda(H.astype(CDT[prec]), torch)
    U = pb.interp(Ht, cuda(X, torch))
    torch.cuda.synchronize()
    ref = sp.interp_direct(sp.half_to_full(H, N, d), X, N)
    assert rel2(to_np(U), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d", [2, 3])
def test_points_on_the_period_boundary_and_on_grid_nodes(lib, torch_mod, prec, d):
    """Coordinates that sit exactly on the period boundary (0, L, -L, 2L, one rounding step
    either side of them), on fine-grid nodes k L / n_f and half-way between nodes, where the
    periodic wrap and the window start round: both transforms still match the direct sums."""
    torch = torch_mod
    N = 16
    nf = 2 * N   # fine grid at sigma = 2 (a multiple of 8 above 2w at both tolerances)
    edge = [0.0, 1.0, -1.0, 2.0, np.nextafter(1.0, 0.0), np.nextafter(0.0, -1.0), np.nextafter(1.0, 2.0),
            -1e-300, 3.0 / nf, 17.0 / nf, (nf - 1.0) / nf, 0.5 / nf, 5.5 / nf, 0.5, -0.5 / nf]
    rng = np.random.default_rng(4242)
    M = 60
    X = np.empty((d, M))
    for a in range(d):
        X[a] = rng.choice(edge, M)
    X[:, 0] = 0.0
    X[:, 1] = np.nextafter(1.0, 0.0)
    F = rng.standard_normal((d, M))
    H = half_random(rng, d, N)
    pb = make(lib, N, d, M, prec)
    fh = pb.spread(cuda(X, torch), cuda(F, torch))
    Hc = H.astype(CDT[prec])
    U = pb.interp(cuda(Hc, torch), cuda(X, torch))
    torch.cuda.synchronize()
    ref = sp.full_to_half(sp.spread_direct(X, F, N), N)
    got = to_np(fh)
    assert rel2(got, ref) <= TOL[prec]
    assert relmax(got, ref) <= 10 * TOL[prec]
    Uref = sp.interp_direct(sp.half_to_full(Hc.astype(np.complex128), N, d), X, N)
    assert rel2(to_np(U), Uref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d", [2, 3])
def test_all_points_at_one_place(lib, torch_mod, prec, d):
    """The densest input the binning can meet: every point at the same position (one bin holds
    them all, so the gather splits the boxes it reaches into the most slices), and a second
    case with the points spread over one fine cell. Both transforms against the direct sums."""
    torch = torch_mod
    N, M = 16, 4000
    rng = np.random.default_rng(99)
    for X in (np.tile(rng.uniform(0, 1, (d, 1)), (1, M)), 0.3 + rng.uniform(0, 1.0 / 32, (d, M))):
        F = rng.standard_normal((d, M))
        H = half_random(rng, d, N)
        pb = make(lib, N, d, M, prec)
        fh = pb.spread(cuda(X, torch), cuda(F, torch))
        Hc = H.astype(CDT[prec])
        U = pb.interp(cuda(Hc, torch), cuda(X, torch))
        torch.cuda.synchronize()
        ref = sp.full_to_half(sp.spread_direct(X, F, N), N)
        got = to_np(fh)
        assert rel2(got, ref) <= TOL[prec]
        assert relmax(got, ref) <= 10 * TOL[prec]
        Uref = sp.interp_direct(sp.half_to_full(Hc.astype(np.complex128), N, d), X, N)
        assert rel2(to_np(U), Uref) <= TOL[prec]


def test_spread_interp_host_pointers_match_device(lib, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(7)
    d, N, M = 3, 12, 333
    X = rng.uniform(0, 1, (d, M))
    F = rng.standard_normal((d, M))
    pb = make(lib, N, d, M, "fp64")
    dev = to_np(pb.spread(cuda(X, torch), cuda(F, torch)))
    host = np.zeros(pb.spec_shape, dtype=np.complex128)
    pb.spread(X, F, None, out=host)
    assert np.array_equal(dev, host) or rel2(host, dev) < 1e-14
    U = np.zeros((d, M))
    pb.interp(host, X, out=U)
    ref = sp.interp_direct(sp.half_to_full(host, N, d), X, N)
    assert rel2(U, ref) <= 1e-10


def test_spread_interp_adjoint(lib, torch_mod):
    """Duality (Sec. 4.4): L^d <f-hat, u-hat> = <c, U> holds for the GPU pair to NUFFT tolerance."""
    torch = torch_mod
    rng = np.random.default_rng(8)
    d, N, M = 3, 16, 400
    X = rng.uniform(0, 1, (d, M))
    c = rng.standard_normal((d, M))
    H = half_random(rng, d, N)
    pb = make(lib, N, d, M, "fp64")
    fh = to_np(pb.spread(cuda(X, torch), cuda(c, torch)))
    U = to_np(pb.interp(cuda(H, torch), cuda(X, torch)))
    lhs = np.sum(sp.half_to_full(fh, N, d) * np.conj(sp.half_to_full(H, N, d))).real
    rhs = np.sum(c * U)
    assert abs(lhs - rhs) <= 1e-10 * np.sum(np.abs(c) * np.abs(U))


# --- fluid updates --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d,N", [(2, 16), (3, 12)])
def test_stokeslet_matches_oracle(lib, torch_mod, prec, d, N):
    torch = torch_mod
    rng = np.random.default_rng(300 + d + N)
    H = half_random(rng, d, N)
    pb = make(lib, N, d, 4, prec, mu=0.7, rho=0.0)
    f = cuda(H.astype(CDT[prec]), torch)
    u = pb.new_spec()
    pb.fluid_step(f, u)
    torch.cuda.synchronize()
    ref = sp.full_to_half(sp.stokeslet(sp.half_to_full(H, N, d), N, 0.7), N)
    got = sp.full_to_half(sp.half_to_full(to_np(u).astype(np.complex128), N, d), N)
    assert rel2(got, ref) <= (1e-6 if prec == "mixed" else 1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp64native", "mixed"])
@pytest.mark.parametrize("d,N", [(2, 16), (2, 10), (3, 8), (3, 12), (3, 48), (3, 96)])
def test_ns_substeps_match_oracle(lib, torch_mod, prec, d, N):
    torch = torch_mod
    rng = np.random.default_rng(400 + d + N)
    mu, rho, dt = 0.05, 1.3, 0.02
    u0 = sp.leray(sp.half_to_full(half_random(rng, d, N), N, d), N)
    f = sp.half_to_full(half_random(rng, d, N), N, d)
    pb = make(lib, N, d, 4, prec, mu=mu, rho=rho, dt=dt)
    cd = CDT[prec]
    ft = cuda(sp.full_to_half(f, N).astype(cd), torch)
    ut = cuda(sp.full_to_half(u0, N).astype(cd), torch)
    uh = pb.new_spec()
    pb.fluid_step(ft, ut, uh)
    torch.cuda.synchronize()
    rh, r1 = sp.ns_substeps(f, u0, N, mu, rho, dt)
    gh = sp.half_to_full(to_np(uh).astype(np.complex128), N, d)
    g1 = sp.half_to_full(to_np(ut).astype(np.complex128), N, d)
    assert rel2(gh, rh) <= TOL[prec]
    assert rel2(g1, r1) <= TOL[prec]
    assert sp.max_divergence(g1, N) <= (1e-6 if prec == "mixed" else 1e-13)


# --- whole steps ------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp64native", "mixed"])
def test_stokes2d_steps_match_oracle(lib, torch_mod, prec):
    """Quasi-static Stokes stepper on a closed elastic curve (the 2D Stokes workload, reduced)."""
    torch = torch_mod
    N, M, dt, nsteps = 32, 128, 1e-3, 5
    rng = np.random.default_rng(1)
    X0 = wl.ellipse(M, 0.3, 0.2, rng.uniform(0, 1, 2))
    pb = make(lib, N, 2, M, prec, mu=1.0, rho=0.0, dt=dt)
    pb.set_force_curve(1.0)
    Xt = cuda(X0, torch)
    pb.step(Xt, nsteps=nsteps)
    torch.cuda.synchronize()
    force = st.curve_model(1.0)
    X = X0.copy()
    for _ in range(nsteps):
        X = st.stokes_step(X, force, N, 1.0, dt)
    disp = X - X0
    assert rel2(to_np(Xt) - X0, disp) <= TOL[prec] * (10 if prec == "mixed" else 1)


@pytest.mark.parametrize("prec", ["fp64", "fp64native", "mixed"])
def test_ns3d_steps_match_oracle(lib, torch_mod, prec):
    torch = torch_mod
    N, dt, nsteps, mu, rho = 12, 2e-3, 2, 0.01, 1.0
    Xref, tri = wl.latlong_sphere(6, 12, 0.25, (0.52, 0.47, 0.5))
    X0 = 0.5 + (Xref - 0.5) * np.array([[1.15], [0.9], [1.0]])
    M = X0.shape[1]
    rng = np.random.default_rng(5)
    u0 = 0.1 * sp.leray(sp.half_to_full(half_random(rng, 3, N), N, 3), N)
    pb = make(lib, N, 3, M, prec, mu=mu, rho=rho, dt=dt)
    pb.set_force_mesh(tri, cuda(Xref, torch), 1.0)
    cd = CDT[prec]
    Xt = cuda(X0, torch)
    ut = cuda(sp.full_to_half(u0, N).astype(cd), torch)
    Ut = pb.interp(ut, Xt)
    pb.step(Xt, ut, Ut, nsteps=nsteps)
    torch.cuda.synchronize()
    force = st.mesh_model(Xref, tri, 1.0)
    X, u = X0.copy(), u0.copy()
    U = sp.interp_direct(u, X, N)
    for _ in range(nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, mu, rho, dt)
    assert rel2(to_np(Xt) - X0, X - X0) <= TOL[prec] * (10 if prec == "mixed" else 1)
    assert rel2(sp.half_to_full(to_np(ut).astype(np.complex128), N, 3), u) <= TOL[prec]
    assert rel2(to_np(Ut), U) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_steps_on_host_buffers_match_device_buffers(lib, torch_mod, prec):
    """fsib_step on host arrays: a single step on a pinned u-hat copies it inside the step
    (beside work that does not read it), pageable arrays and multi-step calls are staged
    around it, and the profiling mode runs the same copies in line. Every form gives the
    device-array result (to rounding: the order of points within a bin is not fixed)."""
    torch = torch_mod
    N, dt, mu, rho = 12, 2e-3, 0.01, 1.0
    Xref, tri = wl.latlong_sphere(6, 12, 0.25, (0.52, 0.47, 0.5))
    X0 = 0.5 + (Xref - 0.5) * np.array([[1.15], [0.9], [1.0]])
    M = X0.shape[1]
    rng = np.random.default_rng(55)
    u0 = sp.full_to_half(0.1 * sp.leray(sp.half_to_full(half_random(rng, 3, N), N, 3), N), N).astype(CDT[prec])
    pb = make(lib, N, 3, M, prec, mu=mu, rho=rho, dt=dt)
    pb.set_force_mesh(tri, cuda(Xref, torch), 1.0)
    U0 = to_np(pb.interp(cuda(u0, torch), cuda(X0, torch)))

    def run(kind, nsteps, profile=False):
        if kind == "device":
            X, u, U = cuda(X0, torch), cuda(u0, torch), cuda(U0, torch)
        elif kind == "pinned":
            X, u, U = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (X0, u0, U0))
        else:
            X, u, U = X0.copy(), u0.copy(), U0.copy()
        pb.profile(profile)
        for _ in range(2):   # twice: the second call replays the captured graph
            pb.step(X, u, U, nsteps=nsteps)
        pb.profile(False)
        torch.cuda.synchronize()
        return [a.detach().cpu().numpy() if hasattr(a, "detach") else a for a in (X, u, U)]

    tol = 1e-12 if prec == "fp64" else 1e-5
    for nsteps in (1, 2):
        ref = run("device", nsteps)
        for kind, prof in (("pinned", False), ("pageable", False), ("pinned", True)):
            got = run(kind, nsteps, prof)
            assert rel2(got[0] - X0, ref[0] - X0) <= tol, (kind, nsteps, prof)
            assert rel2(got[1], ref[1]) <= tol, (kind, nsteps, prof)
            assert rel2(got[2], ref[2]) <= tol, (kind, nsteps, prof)
            assert np.max(np.abs(got[1] - u0)) > 0      # the host u-hat was written back


def test_step_graph_and_direct_agree(lib, torch_mod):
    torch = torch_mod
    N, M = 16, 64
    X0 = wl.ellipse(M, 0.25, 0.2, (0.4, 0.6))
    res = []
    for graph in (True, False):
        pb = make(lib, N, 2, M, "fp64", mu=0.02, rho=1.0, dt=1e-3, graph=graph)
        pb.set_force_curve(1.0)
        X = cuda(X0, torch)
        u = pb.new_spec()
        U = torch.zeros_like(X)
        pb.step(X, u, U, nsteps=3)
        torch.cuda.synchronize()
        res.append(to_np(X))
    assert rel2(res[0] - X0, res[1] - X0) <= 1e-12


# --- invariants -------------------------------------------------------------------------------

def test_invariants_match_oracle(lib, torch_mod):
    torch = torch_mod
    N = 12
    Xref, tri = wl.latlong_sphere(5, 10, 0.25, (0.5, 0.5, 0.5))
    X = 0.5 + (Xref - 0.5) * np.array([[1.1], [0.95], [1.0]])
    M = X.shape[1]
    rng = np.random.default_rng(11)
    H = half_random(rng, 3, N)
    pb = make(lib, N, 3, M, "fp64", mu=0.3, rho=1.7)
    pb.set_force_mesh(tri, Xref, 1.0)
    inv = pb.invariants(cuda(X, torch), cuda(H, torch))
    u = sp.half_to_full(H, N, 3)
    edges, K = lg.spring_stiffness(Xref, tri, 1.0)
    assert abs(inv["volume"] - lg.enclosed_volume(X, tri)) <= 1e-14
    assert abs(inv["Ep"] - lg.spring_energy(X, edges, K)) <= 1e-12 * abs(inv["Ep"])
    assert abs(inv["Ek"] - sp.kinetic_energy(u, N, 1.7)) <= 1e-12 * inv["Ek"]
    assert abs(inv["dissipation"] - sp.dissipation(u, N, 0.3)) <= 1e-12 * inv["dissipation"]
    assert abs(inv["u0"] - np.linalg.norm(u[:, 0, 0, 0])) <= 1e-14
    assert abs(inv["max_div"] - sp.max_divergence(u, N)) <= 1e-12
    # force of the model equals the oracle's spring force
    c = to_np(pb.force(cuda(X, torch)))
    assert rel2(c, lg.spring_force(X, edges, K)) <= 1e-14


def test_nonfinite_is_reported(lib, torch_mod):
    torch = torch_mod
    X = wl.ellipse(32, 0.2, 0.2, (0.5, 0.5))
    X[0, 3] = np.nan
    pb = make(lib, 8, 2, 32, "fp64")
    pb.set_force_curve(1.0)
    with pytest.raises(lib.FsibError) as ei:
        pb.invariants(cuda(X, torch))
    assert ei.value.code == -4


def test_bad_arguments_rejected(lib, torch_mod):
    with pytest.raises(lib.FsibError):
        lib.Problem(7, 3, 10, 1.0, 1.0, 1e-3, 1e-6)      # odd N
    with pytest.raises(lib.FsibError):
        lib.Problem(16, 4, 10, 1.0, 1.0, 1e-3, 1e-6)     # d = 4
    pb = lib.Problem(16, 2, 10, 1.0, 1.0, 1e-3, 1e-6)
    with pytest.raises(lib.FsibError):
        pb.set_option("no_such_key", 1)
    with pytest.raises(lib.FsibError) as ei:
        pb.step(np.zeros((2, 10)), pb.new_spec(), np.zeros((2, 10)))  # no force model
    assert ei.value.code == -7


def test_velocity_guard_after_a_move_beyond_the_widened_bands(lib, torch_mod):
    """The inverse transform behind U^{m+1} computes only the rows within one box of the
    windows at X^{m+1/2}. A uniform flow that carries a cluster of points several boxes in a
    half step (far beyond any stable time step) must give NaN there, never a value read from
    rows that were not computed, and the next call must return FSIB_ENONFINITE; at a normal
    step size the same setup gives the flow speed."""
    torch = torch_mod
    N, d, M = 64, 3, 40          # fine grid 128^3: 16 boxes of 8 cells per axis
    rng = np.random.default_rng(77)
    X0 = rng.uniform(0.45, 0.55, (d, M))
    for dt, expect_nan in ((0.5, True), (1e-3, False)):
        pb = lib.Problem(N, d, M, 0.1, 1.0, dt, 1e-12)
        pb.set_force_target(X0, 0.0, 1.0)              # no boundary force
        u = np.zeros((d, N, N, N), dtype=np.complex128)
        u[1, 0, 0, 0] = 1.0                              # uniform flow u = (0, 1, 0)
        uh = cuda(sp.full_to_half(u, N), torch)
        Xt = cuda(X0, torch)
        Ut = pb.interp(uh, Xt)
        pb.step(Xt, uh, Ut, nsteps=1)
        torch.cuda.synchronize()
        got = to_np(Ut)
        if expect_nan:
            assert np.isnan(got).all()
            # the next call reports it as an error, without running, and clears the record
            with pytest.raises(lib.FsibError) as e:
                pb.step(Xt, uh, Ut, nsteps=1)
            assert e.value.code == -4 and "moved more than one box" in str(e.value)
            assert np.isnan(to_np(Ut)).all()
            pb.interp(uh, Xt, out=Ut)                    # recovers: U^m from the spectrum
            torch.cuda.synchronize()
            assert np.isfinite(to_np(Ut)).all()
            # a synchronous step (host arrays) reports it at once
            Xh, uhh, Uh = X0.copy(), np.ascontiguousarray(sp.full_to_half(u, N)), np.empty_like(X0)
            pb.interp(uhh, Xh, out=Uh)
            with pytest.raises(lib.FsibError) as e:
                pb.step(Xh, uhh, Uh, nsteps=1)
            assert e.value.code == -4
        else:
            assert np.allclose(got[1], 1.0, rtol=0, atol=1e-10)
            assert np.allclose(got[[0, 2]], 0.0, atol=1e-10)
