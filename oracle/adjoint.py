"""Reverse mode of the quasi-static Stokes stepper (oracle).

The boundary velocity is U(X) = interp(G spread(X, c(X)), X): by Eqs.
force_spreading_quad, velo_intp_fini and stokeslet, U_i = sum_j K(X_i - X_j) c_j with
K(r) = L^-d sum_{k in K_N} G(k) exp(i k.r), a real, even, symmetric matrix kernel
(G(k) = mu^-1 (I/|k|^2 - k k^T/|k|^4), G(0) = 0). For a cotangent lam:

  lam . dU = sum_j w_j . dc_j + sum_i dX_i . (grad u(X_i))^T lam_i + sum_j dX_j . (grad w(X_j))^T c_j

with u(x) = sum_j K(x - X_j) c_j (the flow of the forces) and w(x) = sum_i K(x - X_i) lam_i
(the flow of the cotangent used as forces); this is the spread/interp duality of
Sec. 4.4 (Eq. pote_energ_derivative) applied to each factor. For the linear, symmetric
spring laws (Eq. elstic_force_2d, Sec. 6.2.3), (dc/dX)^T w = c(w), and with c = sigma c_1,
lam . dU/dsigma = sum_j w_j . c_j / sigma.

Gradients of the interpolated fields are type-2 sums of i k_b u-hat_a.
"""
from __future__ import annotations

import numpy as np

from . import spectral as sp


def grad_at_points(Fu: np.ndarray, X: np.ndarray, N: int, L: float = 1.0) -> np.ndarray:
    """G[b, a, j] = d u_a / d x_b at X_j, by the type-2 sum of i k_b u-hat_a."""
    d = X.shape[0]
    ks = sp.wavevectors(N, d, L)
    return np.stack([sp.interp_direct(1j * ks[b][None] * Fu, X, N, L) for b in range(d)])


def stokes_velocity_vjp(X, lam, force, sigma, N, mu, L=1.0):
    """(J^T lam, lam . dU/dsigma) for U(X) = interp(stokeslet(spread(X, force(X))), X)."""
    c = force(X)
    u = sp.stokeslet(sp.spread_direct(X, c, N, L), N, mu, L)
    wv = sp.stokeslet(sp.spread_direct(X, lam, N, L), N, mu, L)
    w = sp.interp_direct(wv, X, N, L)
    Gu = grad_at_points(u, X, N, L)
    Gw = grad_at_points(wv, X, N, L)
    gX = np.einsum("baj,aj->bj", Gu, lam) + np.einsum("baj,aj->bj", Gw, c) + force(w)
    gsig = float(np.sum(w * c)) / sigma
    return gX, gsig


def stokes_step_vjp(X, lam1, force, sigma, N, mu, dt, L=1.0):
    """Reverse of X1 = X + dt U(X + dt/2 U(X)) (the midpoint rule of the Stokes stepper)."""
    from .stepper import stokes_velocity
    Xh = X + 0.5 * dt * stokes_velocity(X, force, N, mu, L)
    a, s1 = stokes_velocity_vjp(Xh, lam1, force, sigma, N, mu, L)
    a = dt * a
    b, s2 = stokes_velocity_vjp(X, a, force, sigma, N, mu, L)
    return lam1 + a + 0.5 * dt * b, dt * s1 + 0.5 * dt * s2


def rollout_grad(X0, K, force, sigma, N, mu, dt, dLdXK_fn, L=1.0):
    """Gradient of loss(X^K) with respect to X^0 and sigma by a full reverse sweep."""
    from .stepper import stokes_step
    xs = [X0]
    for _ in range(K):
        xs.append(stokes_step(xs[-1], force, N, mu, dt, L))
    lam = dLdXK_fn(xs[-1])
    gs = 0.0
    for m in range(K - 1, -1, -1):
        lam, s = stokes_step_vjp(xs[m], lam, force, sigma, N, mu, dt, L)
        gs += s
    return lam, gs, xs[-1]


def sphere_loss(X, center, R):
    """sum_j (|X_j - center| - R)^2 and its gradient."""
    D = X - np.asarray(center)[:, None]
    r = np.sqrt(np.sum(D * D, axis=0))
    e = r - R
    return float(np.sum(e * e)), 2.0 * e[None, :] * D / r[None, :]
