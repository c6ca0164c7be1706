"""Pins of the oracle's time steppers against the invariants the paper proves (Sec. 4) and
the closed-form normal-force circle (Sec. 6.1)."""
import math

import numpy as np
import pytest

from oracle import lagrangian as lg
from oracle import spectral as sp
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl


def _phase_shift(Fu, r, N, d):
    ks = sp.wavevectors(N, d)
    return Fu * np.exp(-1j * sum(ks[a] * r[a] for a in range(d)))[None]


def _small_ns2d(N=12, M=40, seed=0):
    rng = np.random.default_rng(seed)
    X = wl.ellipse(M, 0.25, 0.17, (0.43, 0.58))
    H = 0.05 * (rng.standard_normal((2, N, N // 2)) + 1j * rng.standard_normal((2, N, N // 2)))
    u = sp.leray(sp.half_to_full(H, N, 2), N)
    return X, u


# P10: normal-force circle -----------------------------------------------------------------

@pytest.mark.parametrize("N", [4, 8, 16])
def test_normal_force_circle_gives_zero_velocity(N):
    """Outward normal force |F| = 1 on a circle r = L/8 is a gradient, so u = 0 to
    machine precision while h_b < L/N (Sec. 6.1, 'normal' case)."""
    Nb, r, mu = 64, 1 / 8, 1.0
    X = wl.ellipse(Nb, r, r, (0.5, 0.5))
    th = 2 * np.pi * np.arange(Nb) / Nb
    c = (2 * np.pi / Nb) * np.stack([np.cos(th), np.sin(th)])
    U = st.stokes_velocity(X, lambda Y: c, N, mu)
    ct = (2 * np.pi / Nb) * np.stack([-np.sin(th), np.cos(th)])  # tangent case, nonzero flow
    Ut = st.stokes_velocity(X, lambda Y: ct, N, mu)
    assert np.max(np.abs(U)) <= 1e-15 * max(1.0, 1e3 * np.max(np.abs(Ut)))
    assert np.max(np.abs(Ut)) > 1e-3


# P5: exact translation invariance ------------------------------------------------------------

def test_translation_invariance_navier_stokes():
    """Shift X by r and u-hat by exp(-i k.r): every stage is phase-equivariant, so the
    shifted run is the unshifted one moved by r (Sec. 4.2.2), here to rounding."""
    N, mu, rho, dt = 12, 0.02, 1.0, 2e-3
    X, u = _small_ns2d(N)
    force = st.curve_model(1.0)
    U = sp.interp_direct(u, X, N)
    r = np.array([0.0123456, -0.3141592])
    Xr, ur = X + r[:, None], _phase_shift(u, r, N, 2)
    Ur = sp.interp_direct(ur, Xr, N)
    for _ in range(3):
        X, u, U = st.ns_step(X, u, U, force, N, mu, rho, dt)
        Xr, ur, Ur = st.ns_step(Xr, ur, Ur, force, N, mu, rho, dt)
    assert np.max(np.abs(Xr - X - r[:, None])) <= 1e-13
    assert np.max(np.abs(Ur - U)) <= 1e-12 * np.max(np.abs(U))
    assert np.max(np.abs(ur - _phase_shift(u, r, N, 2))) <= 1e-13 * np.max(np.abs(u))


def test_translation_invariance_stokes_3d():
    Xref, tri = wl.latlong_sphere(3, 6, 0.25, (0.5, 0.5, 0.5))
    X0 = Xref * np.array([[1.1], [0.9], [1.0]]) + np.array([[-0.05], [0.05], [0.0]])
    force = st.mesh_model(Xref, tri, 1.0)
    r = np.array([0.17, -0.021, 0.333])
    A = st.stokes_step(X0, force, 6, 1.0, 1e-3)
    B = st.stokes_step(X0 + r[:, None], force, 6, 1.0, 1e-3)
    assert np.max(np.abs(B - A - r[:, None])) <= 1e-14


# P6: momentum ---------------------------------------------------------------------------------

def test_momentum_zero_mode():
    """rho L^d d u-hat(0)/dt = sum_j omega_j F_j (Sec. 4.3): internal forces leave u-hat(0)
    unchanged; a constant external force G per point adds dt * sum(G)/(rho L^d)."""
    N, mu, rho, dt = 12, 0.02, 1.3, 2e-3
    X, u = _small_ns2d(N)
    U = sp.interp_direct(u, X, N)
    inner = st.curve_model(1.0)
    X1, u1, _ = st.ns_step(X, u, U, inner, N, mu, rho, dt)
    assert np.max(np.abs(u1[:, 0, 0] - u[:, 0, 0])) <= 1e-15
    G = np.array([0.3, -0.7])
    ext = lambda Y: inner(Y) + G[:, None] * np.ones(Y.shape[1])
    X2, u2, _ = st.ns_step(X, u, U, ext, N, mu, rho, dt)
    expect = dt * G * X.shape[1] / rho
    assert np.allclose((u2[:, 0, 0] - u[:, 0, 0]).real, expect, atol=1e-15, rtol=1e-13)
    assert np.max(np.abs(u2[:, 0, 0].imag - u[:, 0, 0].imag)) <= 1e-15


# P7 / P14: energy identity and second order in time ------------------------------------------

def test_energy_identity_residual_is_second_order():
    """d(E_K + E_p)/dt = -mu L^d sum |k|^2 |u-hat|^2 (Sec. 4.4, with the L^d factor
    of Eq. kine_energ_derivative). The one-step residual of the scheme shrinks
    like dt^2."""
    N, mu, rho, K = 12, 0.02, 1.0, 1.0
    X, u = _small_ns2d(N)
    force = st.curve_model(K)
    U = sp.interp_direct(u, X, N)
    E0 = sp.kinetic_energy(u, N, rho) + lg.curve_energy(X, K)
    res = []
    for dt in (4e-3, 2e-3, 1e-3):
        X1, u1, _ = st.ns_step(X, u, U, force, N, mu, rho, dt)
        E1 = sp.kinetic_energy(u1, N, rho) + lg.curve_energy(X1, K)
        Dm = 0.5 * (sp.dissipation(u, N, mu) + sp.dissipation(u1, N, mu))
        res.append(abs((E1 - E0) / dt + Dm))
    scale = sp.dissipation(u, N, mu)
    assert res[0] < 0.05 * scale
    assert res[1] < res[0] / 3.0 and res[2] < res[1] / 3.0


def test_second_order_in_time():
    N, mu, rho = 12, 0.02, 1.0
    X0, u0 = _small_ns2d(N)
    force = st.curve_model(1.0)
    T = 8e-3

    def run(nsteps):
        X, u = X0.copy(), u0.copy()
        U = sp.interp_direct(u, X, N)
        for _ in range(nsteps):
            X, u, U = st.ns_step(X, u, U, force, N, mu, rho, T / nsteps)
        return X

    ref = run(32)
    e = [np.max(np.abs(run(n) - ref)) for n in (2, 4, 8)]
    assert e[1] < e[0] / 3.0 and e[2] < e[1] / 3.0


# P4 / P8: divergence-free field, volume ------------------------------------------------------

def test_ns_step_keeps_divergence_free_and_area():
    N, mu, rho, dt = 16, 0.05, 1.0, 1e-3
    X, u = _small_ns2d(N, M=64)
    U = sp.interp_direct(u, X, N)
    force = st.curve_model(1.0)
    for _ in range(5):
        X, u, U = st.ns_step(X, u, U, force, N, mu, rho, dt)
        assert sp.max_divergence(u, N) <= 1e-14


def _area_rate(X, U):
    """Exact d/dt of the polygon area when the vertices move with velocities U."""
    Xp, Xm = np.roll(X, -1, axis=1), np.roll(X, 1, axis=1)
    return 0.5 * float(np.sum(U[0] * (Xp[1] - Xm[1]) - U[1] * (Xp[0] - Xm[0])))


def test_interpolated_velocity_does_not_leak_area():
    """The interpolated field is divergence-free everywhere (Sec. 4.1), so the rate of
    change of the enclosed area vanishes as the boundary is resolved; a field with
    a divergent part keeps a finite leak."""
    N = 12
    _, u = _small_ns2d(N)
    rng = np.random.default_rng(9)
    H = 0.05 * (rng.standard_normal((2, N, N // 2)) + 1j * rng.standard_normal((2, N, N // 2)))
    bad = sp.half_to_full(H, N, 2)  # not projected
    rates, bad_rates = [], []
    for M in (64, 128, 256):
        X = wl.ellipse(M, 0.25, 0.17, (0.43, 0.58))
        rates.append(abs(_area_rate(X, sp.interp_direct(u, X, N))))
        bad_rates.append(abs(_area_rate(X, sp.interp_direct(bad, X, N))))
    # the polygon error of a smooth closed curve decays spectrally: roundoff already at M = 64
    assert max(rates) <= 1e-14 * max(bad_rates)
    assert bad_rates[2] > 0.1
    assert abs(bad_rates[2] - bad_rates[1]) < 0.05 * bad_rates[2]  # finite limit: a real leak


def test_3d_membrane_ns_step_small():
    Xref, tri = wl.latlong_sphere(4, 8, 0.25, (0.5, 0.5, 0.5))
    X = 0.5 + (Xref - 0.5) * np.array([[1.1], [0.9], [1.0]])
    force = st.mesh_model(Xref, tri, 1.0)
    N = 6
    u = np.zeros((3, N, N, N), dtype=complex)
    U = np.zeros_like(X)
    V0 = lg.enclosed_volume(X, tri)
    X1, u1, U1 = st.ns_step(X, u, U, force, N, 0.01, 1.0, 1e-3)
    assert sp.max_divergence(u1, N) <= 1e-14
    assert np.max(np.abs(u1[:, 0, 0, 0])) <= 1e-17
    assert abs(lg.enclosed_volume(X1, tri) / V0 - 1) < 1e-6


# P14 for the quasi-static Stokes stepper (reading C12) ----------------------------------------

def test_stokes_midpoint_step_is_second_order_against_an_ode_solver():
    """The quasi-static Stokes stepper advances dX/dt = U(X), U = interp(Stokeslet(spread(F(X)))),
    by the midpoint rule of Eqs. spatial_1 and spatial_4 (X^{m+1/2} = X^m + dt/2 U(X^m),
    X^{m+1} = X^m + dt U(X^{m+1/2})). Against an independent high-accuracy solution of the same
    ODE (scipy's DOP853 at rtol 1e-13) its error falls by 4 when dt halves. A forward-Euler step,
    a second stage evaluated at X^m, or an average of the two stage velocities would each fall
    by 2, and fail."""
    integrate = pytest.importorskip("scipy.integrate")
    N, M, mu, T = 8, 16, 1.0, 0.05
    X0 = wl.ellipse(M, 0.3, 0.15, (0.47, 0.52))
    force = st.curve_model(1.0)

    def rhs(t, y):
        return st.stokes_velocity(y.reshape(2, M), force, N, mu).ravel()

    ref = integrate.solve_ivp(rhs, (0.0, T), X0.ravel(), method="DOP853", rtol=1e-13,
                              atol=1e-15).y[:, -1].reshape(2, M)
    assert np.linalg.norm(ref - X0) > 1e-3  # the boundary moves well above the errors measured

    def run(step, n):
        X = X0.copy()
        for _ in range(n):
            X = step(X, T / n)
        return X

    def ratios(step):
        e = [np.linalg.norm(run(step, n) - ref) for n in (4, 8, 16, 32)]
        return [e[i] / e[i + 1] for i in range(3)]

    midpoint = ratios(lambda X, dt: st.stokes_step(X, force, N, mu, dt))
    assert all(3.8 < r < 4.2 for r in midpoint), midpoint
    # plausible mistakes, written here, are first order
    euler = ratios(lambda X, dt: X + dt * st.stokes_velocity(X, force, N, mu))
    averaged = ratios(lambda X, dt: X + 0.5 * dt * (st.stokes_velocity(X, force, N, mu) + st.stokes_velocity(
        X + 0.5 * dt * st.stokes_velocity(X, force, N, mu), force, N, mu)))
    for r in (euler, averaged):
        assert all(1.8 < q < 2.2 for q in r), r
