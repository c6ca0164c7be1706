"""Lagrangian part of the oracle: force laws, energies, enclosed area and volume.

Positions are (d, M) float64 arrays, kept unwrapped (differences of positions
are taken without any periodic wrap).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Closed curve with Hookean tension (Eq. elstic_force_2d)
# ---------------------------------------------------------------------------

def curve_weight(M: int) -> float:
    """Quadrature weight omega = d-theta = 2*pi/M of the equispaced curve parameter (Sec. 6.1)."""
    return 2.0 * math.pi / M


def curve_force(X: np.ndarray, K: float) -> np.ndarray:
    """F_i = K (X_{i+1} + X_{i-1} - 2 X_i) / d-theta^2, periodic in i (Eq. elstic_force_2d)."""
    dth = curve_weight(X.shape[1])
    return K * (np.roll(X, -1, axis=1) + np.roll(X, 1, axis=1) - 2.0 * X) / dth ** 2


def curve_energy(X: np.ndarray, K: float) -> float:
    """E_p = K/(2 d-theta) sum_i |X_{i+1} - X_i|^2, so that omega F_i = -dE_p/dX_i."""
    dth = curve_weight(X.shape[1])
    e = np.roll(X, -1, axis=1) - X
    return float(0.5 * K / dth * np.sum(e * e))


def enclosed_area(X: np.ndarray) -> float:
    """Signed area of the closed polygon, (1/2) sum_i (x_i y_{i+1} - x_{i+1} y_i)."""
    x, y = X[0], X[1]
    return float(0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


# ---------------------------------------------------------------------------
# Triangulated membrane with cot-weight springs (Sec. 6.2.3)
# ---------------------------------------------------------------------------

def target_force(X: np.ndarray, Xt: np.ndarray, K: float) -> np.ndarray:
    """Target-point springs F_i = K (X~_i - X_i) that hold wall markers near fixed
    targets (Poiseuille channel, Sec. 5.2.2)."""
    return K * (Xt - X)


def target_energy(X: np.ndarray, Xt: np.ndarray, K: float, omega: float) -> float:
    """E_p = (omega K / 2) sum_i |X~_i - X_i|^2, so that omega F_i = -dE_p/dX_i."""
    return float(0.5 * omega * K * np.sum((Xt - X) ** 2))


def _edge_lengths_sq(X, tri):
    A, B, C = X[:, tri[:, 0]], X[:, tri[:, 1]], X[:, tri[:, 2]]
    a2 = np.sum((B - C) ** 2, axis=0)  # opposite A
    b2 = np.sum((A - C) ** 2, axis=0)  # opposite B
    c2 = np.sum((A - B) ** 2, axis=0)  # opposite C
    return a2, b2, c2


def triangle_areas(X: np.ndarray, tri: np.ndarray) -> np.ndarray:
    A, B, C = X[:, tri[:, 0]], X[:, tri[:, 1]], X[:, tri[:, 2]]
    n = np.cross((B - A).T, (C - A).T)
    return 0.5 * np.sqrt(np.sum(n * n, axis=1))


def spring_stiffness(Xref: np.ndarray, tri: np.ndarray, sigma: float):
    """Edge stiffness from the reference configuration (Sec. 6.2.3).

    For an edge c shared by triangles Delta_c, K_c = sum over Delta_c of
    (sigma/8) (a0^2 + b0^2 - c0^2) / S0, which equals (sigma/2)(cot C1 + cot C2).
    Returns (edges (E, 2) int64 with i < j, K (E,) float64).
    """
    a2, b2, c2 = _edge_lengths_sq(Xref, tri)
    S0 = triangle_areas(Xref, tri)
    acc = {}
    # (edge endpoints, squared length of the edge, squared lengths of the other two)
    for (p, q), e2, o1, o2 in (((0, 1), c2, a2, b2), ((1, 2), a2, b2, c2), ((2, 0), b2, a2, c2)):
        w = sigma / 8.0 * (o1 + o2 - e2) / S0
        for t in range(tri.shape[0]):
            i, j = int(tri[t, p]), int(tri[t, q])
            key = (i, j) if i < j else (j, i)
            acc[key] = acc.get(key, 0.0) + float(w[t])
    keys = sorted(acc)
    edges = np.array(keys, dtype=np.int64).reshape(-1, 2)
    K = np.array([acc[k] for k in keys], dtype=np.float64)
    return edges, K


def spring_force(X: np.ndarray, edges: np.ndarray, K: np.ndarray) -> np.ndarray:
    """F_i = sum_{j linked with i} K_ij (X_j - X_i) (Sec. 6.2.3); nodal forces, omega = 1."""
    F = np.zeros_like(X)
    i, j = edges[:, 0], edges[:, 1]
    D = K[None, :] * (X[:, j] - X[:, i])
    for a in range(X.shape[0]):
        np.add.at(F[a], i, D[a])
        np.add.at(F[a], j, -D[a])
    return F


def spring_energy(X: np.ndarray, edges: np.ndarray, K: np.ndarray) -> float:
    """E = sum_edges (K/2) |X_i - X_j|^2; F = -dE/dX for the force above."""
    e = X[:, edges[:, 0]] - X[:, edges[:, 1]]
    return float(0.5 * np.sum(K * np.sum(e * e, axis=0)))


def membrane_energy(X: np.ndarray, Xref: np.ndarray, tri: np.ndarray, sigma: float) -> float:
    """E = (sigma/2) sum_tri sum_cyc a^2 (b0^2 + c0^2 - a0^2) / (8 S0) (Eq. total_elastic_energy)."""
    a2, b2, c2 = _edge_lengths_sq(X, tri)
    a02, b02, c02 = _edge_lengths_sq(Xref, tri)
    S0 = triangle_areas(Xref, tri)
    s = a2 * (b02 + c02 - a02) + b2 * (a02 + c02 - b02) + c2 * (a02 + b02 - c02)
    return float(0.5 * sigma * np.sum(s / (8.0 * S0)))


def surface_area(X: np.ndarray, tri: np.ndarray) -> float:
    """Area of the triangulated surface: the sum of its triangles' areas (Sec. 6.2.4)."""
    return float(np.sum(triangle_areas(X, tri)))


def surface_tension_force(X: np.ndarray, tri: np.ndarray, gamma: float) -> np.ndarray:
    """Surface tension E = gamma S (Sec. 6.2.4): at node i,
    F_i = -(gamma/2) sum over the triangles (i, j, k) containing i of (X_j - X_k) x n_ijk,
    each triangle's vertices taken in its counter-clockwise order starting at i and
    n_ijk its unit normal by the right-hand rule of (X_i, X_j, X_k). Nodal forces, omega = 1."""
    F = np.zeros_like(X)
    for r in range(3):
        i, j, k = tri[:, r], tri[:, (r + 1) % 3], tri[:, (r + 2) % 3]
        Xi, Xj, Xk = X[:, i].T, X[:, j].T, X[:, k].T
        n = np.cross(Xj - Xi, Xk - Xi)
        n /= np.linalg.norm(n, axis=1)[:, None]
        f = -0.5 * gamma * np.cross(Xj - Xk, n)
        for a in range(3):
            np.add.at(F[a], i, f[:, a])
    return F


def enclosed_volume(X: np.ndarray, tri: np.ndarray) -> float:
    """V = (1/6) sum over ccw triangles (i,j,k) of X_i . (X_j x X_k).

    This is the signed-tetrahedron volume that Sec. 6.2.3 describes; the triple
    product as printed there, of (X_j-X_k, X_k-X_i, X_i-X_j), is identically
    zero because the three vectors sum to zero, so the standard form is used.
    """
    A, B, C = X[:, tri[:, 0]], X[:, tri[:, 1]], X[:, tri[:, 2]]
    return float(np.sum(A * np.cross(B.T, C.T).T) / 6.0)
