"""Pins of the oracle's pressure (Eq. pressure_poisson_k) against closed forms.

Stokes forcing by one sine mode, the Taylor-Green vortex (whose convective term is a pure
gradient), and the circle of Sec. 6.1: a uniform normal force gives zero velocity and a
pressure that is constant inside and outside with the jump F/r (the paper's closed form,
approached as N grows), a uniform tangential force gives no pressure at all.
"""
import math

import numpy as np
import pytest

from oracle import spectral as sp


def _at(p, Y, N):
    return sp.interp_direct(p[None], Y, N)[0]


def test_pressure_of_a_sine_force():
    """f = (sin 2 pi x, 0): Delta p = div f gives p = -cos(2 pi x) / (2 pi)."""
    N = 8
    f = np.zeros((2, N, N), dtype=np.complex128)
    f[0, 0, 1], f[0, 0, N - 1] = -0.5j, 0.5j
    p = sp.pressure(f, None, N, 1.0)
    Y = np.random.default_rng(1).uniform(0, 1, (2, 25))
    assert np.max(np.abs(_at(p, Y, N) + np.cos(2 * math.pi * Y[0]) / (2 * math.pi))) <= 1e-15


def test_pressure_of_the_taylor_green_vortex():
    """u = (sin 2 pi x cos 2 pi y, -cos 2 pi x sin 2 pi y), f = 0: u.grad u = -grad p / rho with
    p = rho (cos 4 pi x + cos 4 pi y) / 4."""
    N, rho = 8, 2.5
    u = np.zeros((2, N, N), dtype=np.complex128)
    for sx in (1, -1):
        for sy in (1, -1):
            # sin(a) cos(b) = sum over the four (±1, ±1) modes of sign / (4i)
            u[0, sy % N, sx % N] = sx / 4j
            u[1, sy % N, sx % N] = -sy / 4j
    Y = np.random.default_rng(2).uniform(0, 1, (2, 30))
    U = sp.interp_direct(u, Y, N)
    assert np.allclose(U[0], np.sin(2 * math.pi * Y[0]) * np.cos(2 * math.pi * Y[1]), atol=1e-15)
    p = sp.pressure(np.zeros_like(u), u, N, rho)
    want = rho * (np.cos(4 * math.pi * Y[0]) + np.cos(4 * math.pi * Y[1])) / 4.0
    assert np.max(np.abs(_at(p, Y, N) - want)) <= 1e-14


def _circle(Nb, r, normal):
    th = 2 * math.pi * np.arange(Nb) / Nb
    X = np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)])
    d = np.stack([np.cos(th), np.sin(th)]) if normal else np.stack([-np.sin(th), np.cos(th)])
    return X, d * (2 * math.pi / Nb)      # force F = 1 per unit theta, weighted by dtheta


def test_normal_circle_pressure_jump():
    """Sec. 6.1: p = (F/r)(pi r^2/L^2) outside, -(F/r)(L^2 - pi r^2)/L^2 inside, u = 0."""
    r, Nb = 0.25, 512
    X, c = _circle(Nb, r, True)
    p_out, p_in = math.pi * r * r / r, -(1.0 - math.pi * r * r) / r
    Y = np.array([[0.5, 0.0], [0.5, 0.0]])       # centre and corner
    errs = []
    for N in (32, 64, 128):
        fh = sp.spread_direct(X, c, N)
        assert np.max(np.abs(sp.stokeslet(fh, N, 1.0))) <= 1e-15
        P = _at(sp.pressure(fh, None, N, 1.0), Y, N)
        errs.append((abs(P[0] - p_in) / abs(p_in), abs(P[1] - p_out) / p_out))
    assert errs[-1][0] < 0.02 and errs[-1][1] < 0.005
    assert errs[0][0] > errs[1][0] > errs[2][0]   # the centre value converges (Gibbs, O(1/N))


def test_tangent_circle_has_no_pressure():
    X, c = _circle(300, 0.3, False)
    N = 32
    p = sp.pressure(sp.spread_direct(X, c, N), None, N, 1.0)
    assert np.max(np.abs(p)) <= 1e-15


def test_pressure_jump_width_is_a_fixed_multiple_of_h():
    """Fig. reso_stokes: with N and N_b refined together the width of the pressure jump
    (height over slope) is a fixed multiple of h, about 2h. Sampled on the Eulerian grid of
    the centreline (slope by central differences over 2h) it settles at 1.70h."""
    r = 0.25
    widths = []
    for N in (32, 64, 128):
        Nb = int(math.ceil(2 * math.pi * r * N))
        X, c = _circle(Nb, r, True)
        p = sp.pressure(sp.spread_direct(X, c, N), None, N, 1.0)
        h = 1.0 / N
        y = np.arange(N) * h
        P = _at(p, np.stack([np.full_like(y, 0.5), y]), N)
        widths.append((1.0 / r) / (np.max(np.abs(P[2:] - P[:-2])) / (2 * h)) / h)
    assert 1.5 < widths[-1] < 2.5
    assert abs(widths[0] - widths[-1]) < 0.02 * widths[-1]


def test_trivial_solutions_vanish_below_the_transition():
    """Sec. 6.1, coupling of L/N and h_b (Fig. circle:error_Nh): with N_b = 64 markers on the
    circle r = L/4 the solutions that should vanish (the normal case's velocity, the tangent
    case's pressure) are at rounding level while the marker spacing h_b = 2 pi r / N_b is
    below the grid spacing h = L/N (N < 41), and are not once it is above it."""
    r, Nb = 0.25, 64
    Xn, cn = _circle(Nb, r, True)
    Xt, ct = _circle(Nb, r, False)
    for N in (8, 16, 32, 48, 64):
        un = np.max(np.abs(sp.stokeslet(sp.spread_direct(Xn, cn, N), N, 1.0)))
        pt = np.max(np.abs(sp.pressure(sp.spread_direct(Xt, ct, N), None, N, 1.0)))
        if 2 * math.pi * r / Nb < 1.0 / N:
            assert un <= 1e-15 and pt <= 1e-13, (N, un, pt)
        else:
            assert un >= 1e-9 and pt >= 1e-7, (N, un, pt)


def test_tangent_circle_is_first_order_when_refined_together():
    """Sec. 6.1 (Fig. u_Nh_h_comp): with N and N_b doubled together (N_b = N / 2, from the
    paper's N = 8, N_b = 4; here the asymptotic range N = 64 .. 512) the velocity of the
    tangent case at the markers converges at first order: successive differences at the
    common markers halve at each refinement."""
    r = 0.25

    def velocity(N, Nb):
        X, c = _circle(Nb, r, False)
        return sp.interp_direct(sp.stokeslet(sp.spread_direct(X, c, N), N, 1.0), X, N)

    U = [velocity(N, N // 2) for N in (64, 128, 256, 512)]
    d = [np.linalg.norm(U[k] - U[k + 1][:, ::2]) / np.linalg.norm(U[k + 1][:, ::2]) for k in range(3)]
    orders = [math.log2(d[k] / d[k + 1]) for k in range(2)]
    assert all(0.9 < q < 1.3 for q in orders), orders
