"""Time steppers of the oracle.

A force model is any callable force(X) -> c returning c_j = omega_j F_j with
shape (d, M), the weighted force that enters the spread of Eq.
force_spreading_quad.
"""
from __future__ import annotations

import numpy as np

from . import lagrangian as lg
from . import spectral as sp


def curve_model(K: float):
    """Closed-curve tension (Eq. elstic_force_2d) weighted by omega = 2*pi/M."""
    def force(X):
        return lg.curve_weight(X.shape[1]) * lg.curve_force(X, K)
    return force


def mesh_model(Xref: np.ndarray, tri: np.ndarray, sigma: float):
    """Cot-weight spring membrane (Sec. 6.2.3); nodal forces, omega = 1."""
    edges, K = lg.spring_stiffness(Xref, tri, sigma)

    def force(X):
        return lg.spring_force(X, edges, K)
    force.edges, force.K = edges, K
    return force


def tension_model(tri: np.ndarray, gamma: float):
    """Surface tension E = gamma S on a triangulated surface (Sec. 6.2.4); nodal forces."""
    def force(X):
        return lg.surface_tension_force(X, tri, gamma)
    return force


def target_model(Xt: np.ndarray, K: float, omega: float):
    """Target-point springs (Sec. 5.2.2) weighted by omega (the Lagrangian meshwidth)."""
    def force(X):
        return omega * lg.target_force(X, Xt, K)
    return force


def add_body_force(fhat: np.ndarray, fbody) -> np.ndarray:
    """Add a uniform body force density f0 (Sec. 5.2.2): its coefficient under
    f-hat(k) = L^-d int f e^{-ik.x} dx is f0 at k = 0 and zero elsewhere."""
    if fbody is None:
        return fhat
    out = fhat.copy()
    d = fhat.shape[0]
    for a in range(d):
        out[(a,) + (0,) * d] += fbody[a]
    return out


def ns_step(X, uhat, U, force, N, mu, rho, dt, L=1.0, Nt=None, fbody=None):
    """One step of Algorithm 1 (Eqs. spatial_1 to spatial_4).

    Inputs: X^m (d, M), full-spectrum u-hat^m, and U^m = u(X^m).
    X^{m+1/2} = X^m + dt/2 U^m; F^{m+1/2} = force(X^{m+1/2}); f-hat by the
    direct type-1 sum; u-hat^{m+1/2} and u-hat^{m+1} by the BE/CN substeps;
    U^{m+1/2} = u^{m+1/2}(X^{m+1/2}); X^{m+1} = X^m + dt U^{m+1/2}; and
    U^{m+1} = u^{m+1}(X^{m+1}), evaluated after the position update (the order
    Algorithm 1 needs, since X^{m+1} must exist first). A uniform body force
    fbody (length d), if given, is added to f-hat.
    Returns (X^{m+1}, u-hat^{m+1}, U^{m+1}).
    """
    Xh = X + 0.5 * dt * U
    c = force(Xh)
    fhat = add_body_force(sp.spread_direct(Xh, c, N, L), fbody)
    uh, u1 = sp.ns_substeps(fhat, uhat, N, mu, rho, dt, L, Nt)
    Uh = sp.interp_direct(uh, Xh, N, L)
    X1 = X + dt * Uh
    U1 = sp.interp_direct(u1, X1, N, L)
    return X1, u1, U1


def stokes_velocity(X, force, N, mu, L=1.0):
    """Quasi-static velocity of the boundary: interp(Stokeslet(spread(force(X), X)), X)."""
    c = force(X)
    fhat = sp.spread_direct(X, c, N, L)
    uhat = sp.stokeslet(fhat, N, mu, L)
    return sp.interp_direct(uhat, X, N, L)


def stokes_step(X, force, N, mu, dt, L=1.0):
    """Midpoint step for quasi-static Stokes: the rule of Eqs. spatial_1 and spatial_4
    with U evaluated from the Stokeslet at X^m and at X^{m+1/2}."""
    U0 = stokes_velocity(X, force, N, mu, L)
    Xh = X + 0.5 * dt * U0
    Uh = stokes_velocity(Xh, force, N, mu, L)
    return X + dt * Uh
