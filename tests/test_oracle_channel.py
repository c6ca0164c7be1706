"""Pins of the oracle's two-dimensional validation pieces (Secs. 5.2.1, 5.2.2).

Target-point springs against their energy, the band flux against a closed form and
against quadrature of the physical field, the body force against exact momentum
balance, the channel's effective boundary width against the paper's figure, and the
integrator's temporal order against the paper's second-order claim.
"""
import math

import numpy as np
import pytest

from oracle import lagrangian as lg
from oracle import spectral as sp
from oracle import stepper as st
import closed_forms as va
from paper_2302_08694_gb300 import workloads as wl


def test_target_force_is_minus_energy_gradient():
    rng = np.random.default_rng(11)
    X = rng.uniform(0, 1, (2, 7))
    Xt = rng.uniform(0, 1, (2, 7))
    K, omega = 3.7, 0.125
    c = st.target_model(Xt, K, omega)(X)
    g = np.zeros_like(X)
    eps = 1e-6
    for a in range(2):
        for j in range(7):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, j] += eps
            Xm[a, j] -= eps
            g[a, j] = (lg.target_energy(Xp, Xt, K, omega) - lg.target_energy(Xm, Xt, K, omega)) / (2 * eps)
    assert np.max(np.abs(c + g)) <= 1e-8 * np.max(np.abs(c))


@pytest.mark.parametrize("y0,y1", [(0.25, 0.75), (0.1, 0.35), (0.0, 1.0), (0.6, 0.2)])
def test_band_flux_of_a_sine_profile(y0, y1):
    """u_x = sin(2 pi y): the flux over [y0, y1] is (cos 2 pi y0 - cos 2 pi y1) / (2 pi)."""
    N = 8
    u = np.zeros((2, N, N), dtype=np.complex128)
    u[0, 1, 0] = -0.5j       # m = (0, 1)
    u[0, N - 1, 0] = 0.5j    # m = (0, -1)
    want = (math.cos(2 * math.pi * y0) - math.cos(2 * math.pi * y1)) / (2 * math.pi)
    assert sp.band_flux(u, N, 0, 1, y0, y1) == pytest.approx(want, abs=1e-15)
    # the other component and the other axis see nothing of this profile
    assert abs(sp.band_flux(u, N, 1, 1, y0, y1)) <= 1e-16
    assert abs(sp.band_flux(u, N, 0, 0, y0, y1)) <= 1e-16


@pytest.mark.parametrize("d,N,comp,axis", [(2, 6, 0, 1), (2, 6, 1, 0), (3, 4, 2, 1), (3, 4, 0, 2), (3, 4, 1, 0)])
def test_band_flux_matches_quadrature_of_the_field(d, N, comp, axis):
    """Average of the physical field over the other axes (uniform rule, exact for the
    kept modes) integrated over the band by Gauss-Legendre."""
    rng = np.random.default_rng(100 + 10 * d + axis)
    u = sp.half_to_full(wl.random_half_spectrum(rng, d, N), N, d)
    y0, y1 = 0.17, 0.71
    gy, gw = np.polynomial.legendre.leggauss(40)
    ys = 0.5 * (y1 - y0) * gy + 0.5 * (y1 + y0)
    ws = 0.5 * (y1 - y0) * gw
    others = [a for a in range(d) if a != axis]
    grid = np.meshgrid(*([np.arange(N) / N] * len(others)), indexing="ij")
    total = 0.0
    for y, w in zip(ys, ws):
        P = np.zeros((d, grid[0].size))
        P[axis] = y
        for a, g in zip(others, grid):
            P[a] = g.ravel()
        total += w * np.mean(sp.interp_direct(u, P, N)[comp])
    assert sp.band_flux(u, N, comp, axis, y0, y1) == pytest.approx(total, rel=1e-12, abs=1e-13)


def test_body_force_alone_accelerates_the_mean_flow():
    """With no boundary force, u-hat(0) grows by dt f0 / rho per step and nothing else moves."""
    N, d = 8, 2
    X = np.array([[0.3, 0.6], [0.4, 0.7]])
    u = np.zeros((d, N, N), dtype=np.complex128)
    U = np.zeros_like(X)
    zero = lambda Y: np.zeros_like(Y)
    f0 = np.array([100.0, -25.0])
    rho, dt = 2.0, 1e-3
    for _ in range(5):
        X, u, U = st.ns_step(X, u, U, zero, N, 0.1, rho, dt, fbody=f0)
    assert np.allclose(u[:, 0, 0], 5 * dt * f0 / rho, rtol=1e-14, atol=0)
    rest = u.copy()
    rest[:, 0, 0] = 0
    assert np.max(np.abs(rest)) == 0.0
    assert np.allclose(U, 5 * dt * f0[:, None] / rho, rtol=1e-13)


def test_momentum_balance_with_target_walls():
    """rho L^d d u-hat(0)/dt = sum_j omega F_j + f0 L^d (Sec. 4 with a body force):
    each step changes u-hat(0) by dt/rho (sum_j c_j(X^{m+1/2}) + f0) exactly."""
    prob = wl.config_poiseuille(N=8)
    ex = prob.extra
    force = st.target_model(ex["Xtarget"], prob.stiffness, ex["omega"])
    rng = np.random.default_rng(5)
    X = prob.X0 + rng.uniform(-0.01, 0.01, prob.X0.shape)
    u = np.zeros((2, 8, 8), dtype=np.complex128)
    U = sp.interp_direct(u, X, 8)
    for _ in range(3):
        Xh = X + 0.5 * prob.dt * U
        want = u[:, 0, 0] + prob.dt / prob.rho * (force(Xh).sum(axis=1) + np.asarray(ex["fbody"]))
        X, u, U = st.ns_step(X, u, U, force, 8, prob.mu, prob.rho, prob.dt, fbody=ex["fbody"])
        assert np.allclose(u[:, 0, 0], want, rtol=1e-12, atol=1e-12)


def _channel_equilibrium(N, T):
    prob = wl.config_poiseuille(N=N, T=T)
    ex = prob.extra
    force = st.target_model(ex["Xtarget"], prob.stiffness, ex["omega"])
    X = prob.X0.copy()
    u = np.zeros((2, N, N), dtype=np.complex128)
    U = np.zeros_like(X)
    for _ in range(prob.nsteps):
        X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, prob.dt, fbody=ex["fbody"])
    y0, y1 = ex["band"]
    return prob, X, sp.band_flux(u, N, 0, 1, y0, y1)


def test_channel_effective_width_follows_the_paper():
    """Fig. effective_width: the FSIB wall is about 0.4 h wide once resolved, the flux
    falls short of Eq. steady_poiseuille_flux, and the wall width shrinks towards that
    value as N grows. At equilibrium the springs carry the body force: the markers sit
    f0 L / (2K) downstream of their targets."""
    widths = {}
    for N in (8, 16):
        prob, X, flux = _channel_equilibrium(N, 2.0)
        ex = prob.extra
        D, f0, h = ex["D"], ex["f0"], 1.0 / N
        steady = va.poiseuille_steady_flux(f0, prob.mu, D)
        assert 0.0 < flux < steady
        widths[N] = (D - va.effective_width(flux, f0, prob.mu)) / h
        shift = f0 * 1.0 / (2 * prob.stiffness)
        assert np.allclose(X[0] - ex["Xtarget"][0], shift, rtol=1e-3)
        assert np.max(np.abs(X[1] - ex["Xtarget"][1])) <= 1e-12
    assert widths[16] < widths[8]
    assert 0.3 < widths[16] < 0.7


def test_sine_circle_is_second_order_in_time():
    """Fig. NS2DerrNt: halving dt divides the velocity error at t = 0.1 by four."""
    N, Nb, T = 16, 50, 0.1
    prob = wl.config_ns2d_circle(N=N, Nb=Nb, T=T)
    u0 = sp.half_to_full(prob.extra["u0"], N, 2)
    force = st.curve_model(prob.stiffness)
    sols = []
    for dt in (0.002, 0.001, 0.0005, 0.000125):
        X, u = prob.X0.copy(), u0.copy()
        U = sp.interp_direct(u, X, N)
        for _ in range(int(round(T / dt))):
            X, u, U = st.ns_step(X, u, U, force, N, prob.mu, prob.rho, dt)
        sols.append(u)
    ref = sols[-1]
    err = [np.linalg.norm(s - ref) / np.linalg.norm(ref) for s in sols[:-1]]
    for a, b in zip(err[:-1], err[1:]):
        assert 3.6 < a / b < 4.6


def test_poiseuille_series_limits():
    """Eq. poiseuille_flux reaches Eq. steady_poiseuille_flux, starts at zero with slope
    f0 D / rho (all fluid accelerates at f0/rho before the walls are felt), and the
    steady flux gives back the channel width."""
    f0, mu, rho, D = 100.0, 0.1, 1.0, 0.5
    steady = va.poiseuille_steady_flux(f0, mu, D)
    assert va.poiseuille_flux(50.0, f0, mu, rho, D)[0] == pytest.approx(steady, rel=1e-9)
    assert va.poiseuille_flux(0.0, f0, mu, rho, D)[0] == 0.0
    t = 1e-6
    slope = va.poiseuille_flux(t, f0, mu, rho, D, nterms=200000)[0] / t
    assert slope == pytest.approx(f0 * D / rho, rel=2e-3)
    assert va.effective_width(steady, f0, mu) == pytest.approx(D, rel=1e-14)
    ts = np.linspace(0.0, 3.0, 31)
    assert np.all(np.diff(va.poiseuille_flux(ts, f0, mu, rho, D)) > 0)


def test_half_spectrum_norm_and_embedding_follow_parseval():
    """The half-spectrum L2 norm equals the field's RMS over a uniform grid (Parseval),
    and embedding in more modes changes neither the field nor its norm."""
    from oracle import spectral as sp
    rng = np.random.default_rng(21)
    for d, N in ((2, 8), (3, 6)):
        H = wl.random_half_spectrum(rng, d, N)
        full = sp.half_to_full(H, N, d)
        H = sp.full_to_half(full, N)           # a consistent (Hermitian, Nyquist-free) half spectrum
        n = 2 * N
        g = np.meshgrid(*([np.arange(n) / n] * d), indexing="ij")
        P = np.stack([gi.ravel() for gi in g[::-1]])
        U = sp.interp_direct(full, P, N)
        rms = math.sqrt(np.mean(np.sum(U * U, axis=0)))
        assert va.half_spectrum_norm(H) == pytest.approx(rms, rel=1e-12)
        E = va.embed_half_spectrum(H, N + 4)
        assert va.half_spectrum_norm(E) == pytest.approx(va.half_spectrum_norm(H), rel=1e-14)
        U2 = sp.interp_direct(sp.half_to_full(E, N + 4, d), P, N + 4)
        assert np.max(np.abs(U2 - U)) <= 1e-12 * np.max(np.abs(U))
    assert va.successive_errors([H, H]) == [0.0]


def test_steady_channel_orders_follow_the_paper():
    """Steady Poiseuille flow with one wall at y = 0 and D = L (Sec. 5.2.2): the wall force that
    balances f0 L^2 is spread from N equispaced markers (omega = h), the Stokeslet gives the
    flow without its mean, and no-slip at the wall fixes the mean. Against
    Eq. steady_poiseuille_velo the error on the grid of the line x = L/2 is first order; with
    the effective width D_e of the computed flux it converges faster, towards the paper's
    order 3/2; Delta_e = D - D_e approaches the 0.4h of Fig. effective_width."""
    mu, f0, L = 0.1, 100.0, 1.0
    e, ee, width = [], [], []
    for N in (16, 32, 64, 128, 256):
        h = L / N
        X = np.stack([np.arange(N) * h, np.zeros(N)])
        F = np.stack([np.full(N, -f0 * L * L / (N * h)), np.zeros(N)])
        u = sp.stokeslet(sp.spread_direct(X, F * h, N), N, mu)
        ubar = -sp.interp_direct(u, X, N)[0].mean()
        yg = np.arange(N) * h
        ug = sp.interp_direct(u, np.stack([np.full(N, 0.5), yg]), N)[0] + ubar
        De = va.effective_width(ubar * L, f0, mu)
        dl = 0.5 * (L - De)
        u_ex = f0 / (2 * mu) * yg * (L - yg)
        u_e = np.where((yg > dl) & (yg < L - dl), f0 / (2 * mu) * (yg - dl) * (L - dl - yg), 0.0)
        e.append(np.linalg.norm(ug - u_ex) / np.linalg.norm(u_ex))
        ee.append(np.linalg.norm(ug - u_e) / np.linalg.norm(u_e))
        width.append((L - De) / h)
        assert abs(ug[0]) <= 1e-9 * np.max(np.abs(ug))    # no slip at the wall
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    orders_e = np.log2(np.array(ee[:-1]) / np.array(ee[1:]))
    assert np.all(np.abs(orders - 1.0) < 0.1)
    assert np.all(orders_e > 1.5) and np.all(np.diff(orders_e) < 0)   # decreasing towards 3/2
    assert 0.40 < width[-1] < 0.42 and np.all(np.diff(width) < 0)
