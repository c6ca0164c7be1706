"""Pins of the oracle's force laws, energies, area and volume."""
import math

import numpy as np
import pytest

from oracle import lagrangian as lg
from paper_2302_08694_gb300 import workloads as wl


def _fd_grad(E, X, eps=1e-6):
    G = np.zeros_like(X)
    for a in range(X.shape[0]):
        for j in range(X.shape[1]):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, j] += eps
            Xm[a, j] -= eps
            G[a, j] = (E(Xp) - E(Xm)) / (2 * eps)
    return G


def test_curve_force_is_energy_gradient_and_sums_to_zero():
    rng = np.random.default_rng(0)
    X = wl.ellipse(24, 0.3, 0.2, (0.4, 0.6)) + 0.01 * rng.standard_normal((2, 24))
    K = 1.7
    F = lg.curve_force(X, K)
    w = lg.curve_weight(24)
    G = _fd_grad(lambda Y: lg.curve_energy(Y, K), X)
    assert np.allclose(w * F, -G, atol=1e-7)       # omega_j F_j = -dE_p/dX_j (Sec. 4.4)
    assert np.max(np.abs(F.sum(axis=1))) <= 1e-10   # net-zero force (Eq. force_vanish)


def test_curve_force_of_circle_points_inward():
    # X = c + r(cos, sin): F = K * (2 cos(dth) - 2) (X - c)/dth^2, a uniform inward normal force
    M, r, K = 32, 0.2, 1.0
    X = wl.ellipse(M, r, r, (0.5, 0.5))
    F = lg.curve_force(X, K)
    dth = 2 * math.pi / M
    ref = K * (2 * math.cos(dth) - 2) / dth ** 2 * (X - 0.5)
    assert np.allclose(F, ref, atol=1e-12)


def test_polygon_area():
    sq = np.array([[0.1, 0.6, 0.6, 0.1], [0.2, 0.2, 0.7, 0.7]])
    assert abs(lg.enclosed_area(sq) - 0.25) <= 1e-15
    assert abs(lg.enclosed_area(sq[:, ::-1]) + 0.25) <= 1e-15
    M = 4096
    X = wl.ellipse(M, 0.3, 0.2, (0.3, 0.9))
    exact = M / 2 * 0.3 * 0.2 * math.sin(2 * math.pi / M)  # affine image of the regular M-gon
    assert abs(lg.enclosed_area(X) - exact) <= 1e-14


@pytest.mark.parametrize("origin", [(0, 0, 0), (0.3, -2.0, 5.0)])
def test_volume_of_cube_is_origin_independent(origin):
    X, tri = wl.cube_mesh(0.7, origin)
    assert abs(lg.enclosed_volume(X, tri) - 0.7 ** 3) <= 1e-14


def test_volume_of_latlong_sphere_converges():
    errs = []
    for n in (10, 20, 40):
        X, tri = wl.latlong_sphere(n, 2 * n, 0.25, (0.1, 0.2, 0.3))
        errs.append(abs(lg.enclosed_volume(X, tri) - 4 / 3 * math.pi * 0.25 ** 3))
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0  # O(h^2)


def test_mesh_is_closed_and_oriented():
    X, tri = wl.latlong_sphere(6, 12, 0.25, (0.5, 0.5, 0.5))
    # every directed edge appears once and its reverse once
    de = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    s = {tuple(e) for e in de}
    assert len(s) == len(de)
    assert all((b, a) in s for a, b in s)
    assert lg.enclosed_volume(X, tri) > 0


def test_cot_spring_stiffness_matches_cotangents():
    X, tri = wl.latlong_sphere(5, 9, 0.25, (0.5, 0.5, 0.5))
    edges, K = lg.spring_stiffness(X, tri, sigma=1.3)
    # (sigma/2)(cot C1 + cot C2) computed from angles
    acc = {}
    for t in tri:
        for p in range(3):
            i, j, k = t[p], t[(p + 1) % 3], t[(p + 2) % 3]
            u, v = X[:, i] - X[:, k], X[:, j] - X[:, k]
            cot = np.dot(u, v) / np.linalg.norm(np.cross(u, v))
            key = (min(i, j), max(i, j))
            acc[key] = acc.get(key, 0.0) + 0.5 * 1.3 * cot
    ref = np.array([acc[(int(a), int(b))] for a, b in edges])
    assert np.allclose(K, ref, rtol=1e-12, atol=1e-12)


def test_membrane_energy_forms_agree_and_force_is_gradient():
    """Eq. total_elastic_energy equals sum_edges K/2 |e|^2 at any deformed state, and
    equals sigma * (reference area) at the reference state (lambda1^2 + lambda2^2 = 2)."""
    rng = np.random.default_rng(4)
    Xref, tri = wl.latlong_sphere(4, 8, 0.25, (0.5, 0.5, 0.5))
    sigma = 0.8
    edges, K = lg.spring_stiffness(Xref, tri, sigma)
    Xd = Xref * np.array([[1.1], [0.95], [1.02]]) + 0.01 * rng.standard_normal(Xref.shape)
    e1 = lg.membrane_energy(Xd, Xref, tri, sigma)
    e2 = lg.spring_energy(Xd, edges, K)
    assert abs(e1 - e2) <= 1e-13 * abs(e1)
    S = lg.triangle_areas(Xref, tri).sum()
    assert abs(lg.membrane_energy(Xref, Xref, tri, sigma) - sigma * S) <= 1e-13
    F = lg.spring_force(Xd, edges, K)
    G = _fd_grad(lambda Y: lg.spring_energy(Y, edges, K), Xd)
    assert np.allclose(F, -G, atol=1e-7)
    assert np.max(np.abs(F.sum(axis=1))) <= 1e-13  # momentum: internal forces sum to zero
