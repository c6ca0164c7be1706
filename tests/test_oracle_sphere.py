"""Pins of the oracle's three-dimensional sphere pieces (Secs. 6.2.3, 6.2.4).

The refined icosahedron against its counting rules and the sphere it approximates, and
the surface-tension force against the gradient of gamma S and two exact identities:
translation invariance (the forces sum to zero) and degree-2 homogeneity of the area
(sum_i X_i . F_i = -2 gamma S, Euler's theorem).
"""
import math

import numpy as np
import pytest

from oracle import lagrangian as lg
from oracle import stepper as st
from paper_2302_08694_gb300 import workloads as wl


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_structure(level):
    R, c = 0.3, np.array([0.4, 0.55, 0.5])
    X, tri = wl.icosphere(level, R, c)
    M, T = X.shape[1], tri.shape[0]
    assert M == 10 * 4 ** level + 2 and T == 20 * 4 ** level
    E = wl.mesh_edges(tri).shape[0]
    assert M - E + T == 2                                   # a topological sphere
    assert np.allclose(np.linalg.norm(X - c[:, None], axis=0), R, rtol=1e-14)
    # consistent orientation: every directed edge appears once and its reverse once
    d = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    s = set(map(tuple, d))
    assert len(s) == 3 * T and all((b, a) in s for a, b in s)
    assert lg.enclosed_volume(X, tri) > 0                   # counter-clockwise from outside


def test_icosphere_converges_to_the_sphere():
    R = 1.0 / 3.0
    errs = []
    for level in (2, 3, 4):
        X, tri = wl.icosphere(level, R, (0.5, 0.5, 0.5))
        errs.append(abs(lg.enclosed_volume(X, tri) / (4.0 / 3.0 * math.pi * R ** 3) - 1.0))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5   # O(h^2)


def _perturbed(level, seed):
    X, tri = wl.icosphere(level, 0.3, (0.5, 0.45, 0.6))
    rng = np.random.default_rng(seed)
    return X + rng.uniform(-0.02, 0.02, X.shape), tri


def test_surface_tension_is_minus_area_gradient():
    X, tri = _perturbed(1, 3)
    gamma = 1.7
    F = lg.surface_tension_force(X, tri, gamma)
    G = np.zeros_like(X)
    eps = 1e-6
    for a in range(3):
        for j in range(X.shape[1]):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, j] += eps
            Xm[a, j] -= eps
            G[a, j] = gamma * (lg.surface_area(Xp, tri) - lg.surface_area(Xm, tri)) / (2 * eps)
    assert np.max(np.abs(F + G)) <= 1e-8 * np.max(np.abs(F))


@pytest.mark.parametrize("level", [1, 3])
def test_surface_tension_identities(level):
    X, tri = _perturbed(level, 4 + level)
    gamma = 0.8
    F = lg.surface_tension_force(X, tri, gamma)
    S = lg.surface_area(X, tri)
    assert np.max(np.abs(F.sum(axis=1))) <= 1e-13 * np.max(np.abs(F)) * X.shape[1]
    assert np.sum(X * F) == pytest.approx(-2.0 * gamma * S, rel=1e-13)
    # on the unperturbed sphere the net force per vertex points inwards
    Xs, _ = wl.icosphere(level, 0.3, (0.5, 0.45, 0.6))
    Fs = lg.surface_tension_force(Xs, tri, gamma)
    radial = np.sum(Fs * (Xs - np.array([[0.5], [0.45], [0.6]])), axis=0)
    assert np.all(radial < 0)


def test_tension_model_matches_the_force():
    X, tri = _perturbed(2, 9)
    assert np.array_equal(st.tension_model(tri, 1.3)(X), lg.surface_tension_force(X, tri, 1.3))


def test_sine_velocity_3d_is_the_stated_field():
    """u_0 = (sin 2 pi z, 0, sin 2 pi y): evaluate the half spectrum at points by the oracle."""
    from oracle import spectral as sp
    N = 8
    u = sp.half_to_full(wl.sine_velocity_half_3d(N), N, 3)
    rng = np.random.default_rng(2)
    P = rng.uniform(0, 1, (3, 20))
    U = sp.interp_direct(u, P, N)
    want = np.stack([np.sin(2 * math.pi * P[2]), np.zeros(20), np.sin(2 * math.pi * P[1])])
    assert np.max(np.abs(U - want)) <= 1e-14
