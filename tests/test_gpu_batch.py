"""Batched problems (one graph launch advances every member) and the autotuner."""
import numpy as np
import pytest

from oracle import spectral as sp
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_problems():
    probs = []
    for i, (d, N, M) in enumerate([(2, 16, 64), (3, 12, 0), (2, 24, 150), (3, 16, 0), (2, 32, 33), (2, 16, 90),
                                   (3, 12, 0)]):
        if d == 2:
            X0 = wl.ellipse(M, 0.25 + 0.01 * i, 0.18, (0.4 + 0.03 * i, 0.55))
            probs.append(dict(d=2, N=N, M=M, X0=X0, force="curve"))
        else:
            Xref, tri = wl.latlong_sphere(4 + i, 8 + 2 * i, 0.25, (0.5, 0.48, 0.51))
            X0 = 0.5 + (Xref - 0.5) * np.array([[1.1], [0.93], [1.0]])
            probs.append(dict(d=3, N=N, M=X0.shape[1], X0=X0, force="mesh", Xref=Xref, tri=tri))
    return probs


def setup(pb, p, torch):
    if p["force"] == "curve":
        pb.set_force_curve(1.0)
    else:
        pb.set_force_mesh(p["tri"], torch.from_numpy(p["Xref"]).cuda(), 1.0)


@pytest.mark.parametrize("merge", [1, 0])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_individual_handles(lib, torch_mod, prec, merge):
    """Both batch graphs (one launch per phase over the members, or one branch per member)
    give every member the result of its own handle."""
    torch = torch_mod
    probs = small_problems()
    n = len(probs)
    tol = 1e-12 if prec == "fp64" else 1e-6
    B = lib.Batch([p["N"] for p in probs], [p["d"] for p in probs], [p["M"] for p in probs],
                  [0.02] * n, [1.0] * n, [2e-3] * n, [tol] * n, precision=prec)
    B.set_option("merge", merge)
    Xb, ub, Ub, singles = [], [], [], []
    for p, m in zip(probs, B.members):
        setup(m, p, torch)
        X = torch.from_numpy(p["X0"].copy()).cuda()
        Xb.append(X)
        ub.append(m.new_spec())
        Ub.append(torch.zeros_like(X))
        s = lib.Problem(p["N"], p["d"], p["M"], 0.02, 1.0, 2e-3, tol, precision=prec)
        setup(s, p, torch)
        singles.append((s, X.clone(), s.new_spec(), torch.zeros_like(X)))
    B.step(Xb, ub, Ub, nsteps=3)
    for s, X, u, U in singles:
        s.step(X, u, U, nsteps=3)
    torch.cuda.synchronize()
    own = sum(s.info("launches_per_step") for s, _, _, _ in singles)
    if merge:
        # members of a group share their launches: fewer kernels than the members' own graphs
        assert B.info("groups") == len({(p["d"], p["N"]) for p in probs})
        assert B.info("launches_per_step") < own
    else:
        # one branch per member: as many kernels as the members' own graphs
        assert B.info("launches_per_step") == own
    t = 1e-12 if prec == "fp64" else 1e-5
    for i, (p, (s, X, u, U)) in enumerate(zip(probs, singles)):
        x0 = p["X0"]
        assert rel2(Xb[i].cpu().numpy() - x0, X.cpu().numpy() - x0) <= t, i
        assert rel2(ub[i].cpu().numpy(), u.cpu().numpy()) <= t, i
    # and one member against the oracle
    p = probs[0]
    force = st.curve_model(1.0)
    X, u, U = p["X0"].copy(), np.zeros((2, p["N"], p["N"]), complex), np.zeros_like(p["X0"])
    for _ in range(3):
        X, u, U = st.ns_step(X, u, U, force, p["N"], 0.02, 1.0, 2e-3)
    assert rel2(Xb[0].cpu().numpy() - p["X0"], X - p["X0"]) <= (1e-10 if prec == "fp64" else 1e-4)
    B.close()


def test_autotune_keeps_results(lib, torch_mod):
    torch = torch_mod
    Xref, tri = wl.latlong_sphere(10, 20, 0.25, (0.5, 0.5, 0.5))
    X0 = 0.5 + (Xref - 0.5) * np.array([[1.1], [0.95], [1.0]])
    M = X0.shape[1]
    res = []
    for tune in (False, True):
        pb = lib.Problem(24, 3, M, 0.01, 1.0, 1e-3, 1e-12)
        pb.set_force_mesh(tri, Xref, 1.0)
        X = torch.from_numpy(X0.copy()).cuda()
        u = pb.new_spec()
        U = torch.zeros_like(X)
        if tune:
            choice = pb.autotune(X, u, U)
            assert choice["fft_tile"] in (4, 8, 16) and choice["fft_rows"] in (2, 4, 8)
            assert np.array_equal(X.cpu().numpy(), X0)  # autotune does not touch the state
        pb.step(X, u, U, nsteps=2)
        torch.cuda.synchronize()
        res.append((X.cpu().numpy(), u.cpu().numpy()))
    assert rel2(res[1][0] - X0, res[0][0] - X0) <= 1e-12
    assert rel2(res[1][1], res[0][1]) <= 1e-12


# Members shaped like the batched workload (2D ellipses and 3D lat-long ellipsoids, mu = 0.01,
# rho = 1, dt = 1e-4), two per (d, N) class so that classes hold several members, N up to 96
# and M in the thousands.
BATCH_SPECS = [(2, 64, 3000), (3, 64, 2000), (2, 64, 1500), (3, 64, 800), (3, 32, 500), (2, 96, 4000)]
_ORACLE = {}


def batch_members():
    out = []
    for i, (d, N, M) in enumerate(BATCH_SPECS):
        prng = np.random.default_rng(3000 + i)
        if d == 2:
            a, b = prng.uniform(0.15, 0.35, 2)
            X0 = wl.ellipse(M, a, b, prng.uniform(0.0, 1.0, 2))
            out.append(dict(d=2, N=N, M=M, X0=X0, force="curve"))
        else:
            n_r = max(2, int(round(np.sqrt((M - 2) / 2.0))))
            c = np.array([0.5, 0.5, 0.5]) + prng.uniform(-0.5 / N, 0.5 / N, 3)
            axes = 0.25 * (1.0 + 0.2 * prng.uniform(-1.0, 1.0, 3))
            Xref, tri = wl.latlong_sphere(n_r, 2 * n_r, 0.25, c)
            X0 = c[:, None] + (Xref - c[:, None]) * (axes / 0.25)[:, None]
            out.append(dict(d=3, N=N, M=X0.shape[1], X0=X0, force="mesh", Xref=Xref, tri=tri))
    return out


def oracle_two_steps(i, p):
    """X, full-spectrum u-hat and U = u(X) after two oracle steps (Algorithm 1) from rest."""
    if i not in _ORACLE:
        force = st.curve_model(1.0) if p["force"] == "curve" else st.mesh_model(p["Xref"], p["tri"], 1.0)
        d, N = p["d"], p["N"]
        X, u, U = p["X0"].copy(), np.zeros((d,) + (N,) * d, complex), np.zeros_like(p["X0"])
        for _ in range(2):
            X, u, U = st.ns_step(X, u, U, force, N, 0.01, 1.0, 1e-4)
        _ORACLE[i] = (X, u, U)
    return _ORACLE[i]


@pytest.mark.parametrize("merge", [1, 0])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_members_match_oracle(lib, torch_mod, prec, merge):
    """Every member of an uneven batch (2D and 3D, N = 32 to 96, M = 500 to 4000) after two
    batched steps, element by element against the oracle: the velocity at the points and the
    full velocity spectrum at the parity tolerance of the precision (relative 2-norm), and the
    positions to a few units in the last place of FP64 plus dt |U| times that tolerance (the
    displacement of two steps of 1e-4 is near the rounding of the positions themselves, so it
    is not compared relatively)."""
    torch = torch_mod
    probs = batch_members()
    n = len(probs)
    tol = 1e-12 if prec == "fp64" else 1e-6
    B = lib.Batch([p["N"] for p in probs], [p["d"] for p in probs], [p["M"] for p in probs],
                  [0.01] * n, [1.0] * n, [1e-4] * n, [tol] * n, precision=prec)
    B.set_option("merge", merge)
    Xb, ub, Ub = [], [], []
    for p, m in zip(probs, B.members):
        setup(m, p, torch)
        X = torch.from_numpy(p["X0"].copy()).cuda()
        Xb.append(X)
        ub.append(m.new_spec())
        Ub.append(torch.zeros_like(X))
    B.step(Xb, ub, Ub, nsteps=2)
    torch.cuda.synchronize()
    t = 1e-10 if prec == "fp64" else 1e-5
    for i, p in enumerate(probs):
        Xo, uo, Uo = oracle_two_steps(i, p)
        eU = rel2(Ub[i].cpu().numpy(), Uo)
        eu = rel2(sp.half_to_full(ub[i].cpu().numpy().astype(np.complex128), p["N"], p["d"]), uo)
        eX = float(np.max(np.abs(Xb[i].cpu().numpy() - Xo)))
        assert eU <= t and eu <= t, (i, p["d"], p["N"], p["M"], eU, eu)
        assert eX <= 4e-16 + 2e-4 * t * np.max(np.abs(Uo)), (i, eX)
    B.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_with_stokes_members_and_group_splits(lib, torch_mod, prec):
    """Quasi-static Stokes members (whose step ends with copies of U and u-hat, recorded like
    the kernels) beside Navier-Stokes members, in groups that group_max splits: every member
    matches its own handle after three steps, whatever the grouping."""
    torch = torch_mod
    specs = [(2, 16, 120, 0.0), (2, 16, 90, 0.0), (2, 16, 70, 0.0), (3, 12, 0, 0.0), (3, 12, 0, 0.0),
             (2, 16, 100, 1.0), (3, 12, 0, 1.0)]
    probs = []
    for i, (d, N, M, rho) in enumerate(specs):
        if d == 2:
            X0 = wl.ellipse(M, 0.22 + 0.01 * i, 0.17, (0.45 + 0.02 * i, 0.52))
            probs.append(dict(d=2, N=N, M=M, X0=X0, force="curve", rho=rho))
        else:
            Xref, tri = wl.latlong_sphere(4 + i % 2, 8 + 2 * (i % 2), 0.25, (0.5, 0.48, 0.51))
            X0 = 0.5 + (Xref - 0.5) * np.array([[1.1], [0.93], [1.0]])
            probs.append(dict(d=3, N=N, M=X0.shape[1], X0=X0, force="mesh", Xref=Xref, tri=tri, rho=rho))
    n = len(probs)
    tol = 1e-12 if prec == "fp64" else 1e-6
    refs = []
    for p in probs:
        s = lib.Problem(p["N"], p["d"], p["M"], 0.02, p["rho"], 2e-3, tol, precision=prec)
        setup(s, p, torch)
        X = torch.from_numpy(p["X0"].copy()).cuda()
        u, U = s.new_spec(), torch.zeros_like(X)
        s.step(X, u, U, nsteps=3)
        torch.cuda.synchronize()
        refs.append((X.cpu().numpy(), u.cpu().numpy(), U.cpu().numpy()))
    t = 1e-12 if prec == "fp64" else 1e-5
    for gmax in (0, 2, 1):
        B = lib.Batch([p["N"] for p in probs], [p["d"] for p in probs], [p["M"] for p in probs], [0.02] * n,
                      [p["rho"] for p in probs], [2e-3] * n, [tol] * n, precision=prec)
        B.set_option("group_max", gmax)
        assert B.info("group_max") == gmax
        Xb, ub, Ub = [], [], []
        for p, m in zip(probs, B.members):
            setup(m, p, torch)
            X = torch.from_numpy(p["X0"].copy()).cuda()
            Xb.append(X)
            ub.append(m.new_spec())
            Ub.append(torch.zeros_like(X))
        B.step(Xb, ub, Ub, nsteps=3)
        torch.cuda.synchronize()
        # 2D Stokes / 3D Stokes / 2D NS / 3D NS classes; group_max splits the three 2D Stokes members
        expect = {0: 4, 2: 5, 1: n}[gmax]
        assert B.info("groups") == expect
        for i, (p, (Xr, ur, Ur)) in enumerate(zip(probs, refs)):
            x0 = p["X0"]
            assert rel2(Xb[i].cpu().numpy() - x0, Xr - x0) <= t, (gmax, i)
            assert rel2(ub[i].cpu().numpy(), ur) <= t, (gmax, i)
            assert rel2(Ub[i].cpu().numpy(), Ur) <= t, (gmax, i)
        B.close()


def test_batch_options_are_checked(lib, torch_mod):
    B = lib.Batch([8, 8], [2, 2], [20, 30], [0.1, 0.1], [1.0, 1.0], [1e-3, 1e-3], [1e-6, 1e-6], precision="mixed")
    assert B.info("merge") == 1 and B.info("group_max") == 0
    for key, value in (("merge", 2), ("group_max", -1), ("group_max", 1.5), ("no_such_key", 1)):
        with pytest.raises(lib.FsibError):
            B.set_option(key, value)
    B.close()
