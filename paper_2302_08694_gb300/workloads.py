"""Seeded synthetic inputs for the FSIB time step.

This module builds boundary geometries, meshes and random test data. It holds
none of the method's arithmetic (no Fourier sums, no force laws, no fluid
solve): both the CUDA path and the CPU oracle consume what it returns.

Geometries follow the paper's own experiments: a closed curve sampled at
equispaced parameter values (Sec. 6.1 and 6.2.1, theta_j = j * 2*pi/N_b) and a
triangulated sphere (Sec. 6.2.3). The paper refines an icosahedron; the
workloads here use a latitude-longitude triangulation instead, which gives the
exact point counts of the benchmark configurations (M = 2 + n_r * n_phi).

All arrays are float64 / int32 NumPy arrays. Positions are structure-of-arrays
with shape (d, M): row a holds coordinate a (0 = x, 1 = y, 2 = z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

L_BOX = 1.0


def ellipse(M: int, a: float, b: float, center) -> np.ndarray:
    """Closed curve X_j = c + (a cos th_j, b sin th_j), th_j = 2*pi*j/M (Sec. 6.1)."""
    th = 2.0 * math.pi * np.arange(M, dtype=np.float64) / M
    X = np.empty((2, M), dtype=np.float64)
    X[0] = center[0] + a * np.cos(th)
    X[1] = center[1] + b * np.sin(th)
    return X


def latlong_sphere(n_r: int, n_phi: int, radius: float, center):
    """Latitude-longitude triangulation of a sphere.

    Vertices: north pole (index 0), n_r interior rings of n_phi points at polar
    angles pi*i/(n_r+1), i = 1..n_r, and the south pole (index M-1).
    Triangles are listed counter-clockwise when seen from outside, so that every
    edge is traversed in opposite directions by its two triangles (the
    orientation rule stated with the volume formula of Sec. 6.2.3).

    Returns (X (3, M) float64, tri (ntri, 3) int32).
    """
    M = 2 + n_r * n_phi
    X = np.empty((3, M), dtype=np.float64)
    X[:, 0] = (center[0], center[1], center[2] + radius)
    X[:, M - 1] = (center[0], center[1], center[2] - radius)
    th = math.pi * np.arange(1, n_r + 1, dtype=np.float64) / (n_r + 1)
    ph = 2.0 * math.pi * np.arange(n_phi, dtype=np.float64) / n_phi
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    X[0, 1:M - 1] = (center[0] + radius * st * np.cos(ph)[None, :]).ravel()
    X[1, 1:M - 1] = (center[1] + radius * st * np.sin(ph)[None, :]).ravel()
    X[2, 1:M - 1] = (center[2] + radius * ct * np.ones_like(ph)[None, :]).ravel()

    def v(i, j):  # ring i in 0..n_r-1, longitude j (wrapped)
        return 1 + i * n_phi + (j % n_phi)

    tris = []
    for j in range(n_phi):  # north fan
        tris.append((0, v(0, j), v(0, j + 1)))
    for i in range(n_r - 1):  # quads split along a fixed diagonal
        for j in range(n_phi):
            a, b = v(i, j), v(i, j + 1)
            c, d = v(i + 1, j), v(i + 1, j + 1)
            tris.append((a, c, d))
            tris.append((a, d, b))
    for j in range(n_phi):  # south fan
        tris.append((M - 1, v(n_r - 1, j + 1), v(n_r - 1, j)))
    return X, np.asarray(tris, dtype=np.int32)


def icosphere(level: int, radius: float, center):
    """Refined icosahedron on a sphere (Sec. 6.2.3).

    Start from the regular icosahedron (12 vertices, 20 triangles); each refinement
    splits every triangle into four through its edge midpoints and projects the new
    vertices onto the sphere, so M = 10 * 4^level + 2 (2562 at level 4, 10242 at 5,
    40962 at 6). Triangles are counter-clockwise seen from outside.

    Returns (X (3, M) float64, tri (ntri, 3) int32).
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    P = [np.asarray(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
         (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                m = P[a] + P[b]
                P.append(m / np.linalg.norm(m))
                mid[key] = len(P) - 1
            return mid[key]
        G = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            G += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = G
    X = np.asarray(center, dtype=np.float64)[:, None] + radius * np.stack(P, axis=1)
    tri = np.asarray(F, dtype=np.int32)
    # orient counter-clockwise from outside: the normal must point away from the centre
    A, B, C = X[:, tri[:, 0]], X[:, tri[:, 1]], X[:, tri[:, 2]]
    n = np.cross((B - A).T, (C - A).T)
    out = np.sum(n * (A - np.asarray(center, dtype=np.float64)[:, None]).T, axis=1)
    flip = out < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return X, tri


def mesh_edges(tri: np.ndarray) -> np.ndarray:
    """Unique undirected edges (E, 2) int32 of a triangle list, sorted (i < j)."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int32)


def cube_mesh(side: float, origin):
    """Unit-cube surface, 12 triangles, counter-clockwise from outside."""
    o = np.asarray(origin, dtype=np.float64)
    P = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                  [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.float64)
    X = (o[None, :] + side * P).T.copy()
    tri = np.array([[0, 2, 1], [0, 3, 2],   # z = 0, normal -z
                    [4, 5, 6], [4, 6, 7],   # z = 1, normal +z
                    [0, 1, 5], [0, 5, 4],   # y = 0, normal -y
                    [3, 7, 6], [3, 6, 2],   # y = 1, normal +y
                    [0, 4, 7], [0, 7, 3],   # x = 0, normal -x
                    [1, 2, 6], [1, 6, 5]],  # x = 1, normal +x
                   dtype=np.int32)
    return X, tri


def random_points(rng: np.random.Generator, d: int, M: int, lo=0.0, hi=L_BOX) -> np.ndarray:
    return rng.uniform(lo, hi, size=(d, M))


def random_force(rng: np.random.Generator, d: int, M: int) -> np.ndarray:
    return rng.standard_normal(size=(d, M))


def random_half_spectrum(rng: np.random.Generator, d: int, N: int, scale=1.0) -> np.ndarray:
    """Random complex array in the library's half-spectrum layout.

    Shape (d, N, N, N//2) for d = 3 and (d, N, N//2) for d = 2, complex128.
    Any complex array is a valid input of that layout; the layout's rules
    (Hermitian part of the m_x = 0 plane, Nyquist entries ignored) decide
    what field it represents.
    """
    shape = (d,) + (N,) * (d - 1) + (N // 2,)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


# ---------------------------------------------------------------------------
# Benchmark configurations (periodic unit box, L = 1)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    d: int
    N: int
    M: int
    mu: float
    rho: float          # rho <= 0 selects the quasi-static Stokes stepper
    dt: float
    nsteps: int
    tol: float
    precision: str      # "fp64" or "mixed"
    force: str          # "curve" (closed-curve tension) or "mesh" (cot-weight springs)
    X0: np.ndarray
    stiffness: float    # K for "curve", sigma for "mesh"
    tri: np.ndarray | None = None
    Xref: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def config_stokes2d(seed: int = 1, N: int = 64, M: int = 256) -> Problem:
    """2D Stokes, FP64: ellipse (0.3, 0.2) at a seeded centre, K = 1, mu = 1."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, 2)
    X0 = ellipse(M, 0.3, 0.2, c)
    return Problem("stokes2d_N64_M256_fp64", 2, N, M, 1.0, 0.0, 1e-4, 200, 1e-12,
                   "fp64", "curve", X0, 1.0)


def _membrane(seed: int, N: int, n_r: int, n_phi: int):
    rng = np.random.default_rng(seed)
    h = L_BOX / N
    c = np.array([0.5, 0.5, 0.5]) + rng.uniform(-h / 2, h / 2, 3)
    axes = 0.25 * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, 3))
    Xref, tri = latlong_sphere(n_r, n_phi, 0.25, c)
    X0 = c[:, None] + (Xref - c[:, None]) * (axes / 0.25)[:, None]
    return Xref, X0, tri


def config_ns3d_fp64(seed: int = 2, N: int = 64, n_r: int = 70, n_phi: int = 144,
                     nsteps: int = 100) -> Problem:
    """3D Navier-Stokes, FP64: lat-long membrane (M = 10082), rho = 1, mu = 0.01."""
    Xref, X0, tri = _membrane(seed, N, n_r, n_phi)
    M = X0.shape[1]
    return Problem(f"ns3d_N{N}_M{M}_fp64", 3, N, M, 0.01, 1.0, 1e-4, nsteps, 1e-12,
                   "fp64", "mesh", X0, 1.0, tri=tri, Xref=Xref)


def config_ns3d_mixed(seed: int = 3, N: int = 128, n_r: int = 140, n_phi: int = 288,
                      nsteps: int = 100) -> Problem:
    """3D Navier-Stokes, FP32-mixed: N = 128, M = 40322, tol 1e-6."""
    Xref, X0, tri = _membrane(seed, N, n_r, n_phi)
    M = X0.shape[1]
    return Problem(f"ns3d_N{N}_M{M}_mixed", 3, N, M, 0.01, 1.0, 1e-4, nsteps, 1e-6,
                   "mixed", "mesh", X0, 1.0, tri=tri, Xref=Xref)


def config_stokes3d_adjoint(seed: int = 5, N: int = 96, n_r: int = 100, n_phi: int = 200) -> Problem:
    """3D Stokes for the differentiable workload: N = 96, M = 20002, mu = 1."""
    Xref, X0, tri = _membrane(seed, N, n_r, n_phi)
    M = X0.shape[1]
    return Problem(f"stokes3d_N{N}_M{M}_mixed", 3, N, M, 1.0, 0.0, 1e-4, 50, 1e-6,
                   "mixed", "mesh", X0, 1.0, tri=tri, Xref=Xref,
                   extra={"ckpt_every": 10, "target_radius": 0.25})


def config_batched(seed: int = 4, nprob: int = 64):
    """64 independent problems, 2D/3D mixed, N in {32,48,64,96,128}, M in [128, 20000]."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(nprob):
        d = 2 if rng.uniform() < 0.5 else 3
        N = int(rng.choice([32, 48, 64, 96, 128]))
        Mt = int(rng.integers(128, 20001))
        prng = np.random.default_rng(1000 + i)
        if d == 2:
            a, b = prng.uniform(0.15, 0.35, 2)
            c = prng.uniform(0.0, 1.0, 2)
            X0 = ellipse(Mt, a, b, c)
            probs.append(Problem(f"b{i}_2d", 2, N, Mt, 0.01, 1.0, 1e-4, 1, 1e-6, "mixed",
                                 "curve", X0, 1.0))
        else:
            n_r = max(2, int(round(math.sqrt(max(Mt - 2, 8) / 2.0))))
            n_phi = 2 * n_r
            h = L_BOX / N
            c = np.array([0.5, 0.5, 0.5]) + prng.uniform(-h / 2, h / 2, 3)
            axes = 0.25 * (1.0 + 0.2 * prng.uniform(-1.0, 1.0, 3))
            Xref, tri = latlong_sphere(n_r, n_phi, 0.25, c)
            X0 = c[:, None] + (Xref - c[:, None]) * (axes / 0.25)[:, None]
            probs.append(Problem(f"b{i}_3d", 3, N, X0.shape[1], 0.01, 1.0, 1e-4, 1, 1e-6,
                                 "mixed", "mesh", X0, 1.0, tri=tri, Xref=Xref))
    return probs


# ---------------------------------------------------------------------------
# Two-dimensional Navier-Stokes validation workloads (Secs. 5.2.1, 5.2.2)
# ---------------------------------------------------------------------------

def sine_velocity_half(N: int) -> np.ndarray:
    """Initial velocity u_0 = (0, sin(2 pi x / L)) in the half-spectrum layout (d = 2).

    sin(2 pi x) = (e^{2 pi i x} - e^{-2 pi i x}) / (2i): the y component holds
    -i/2 at m = (1, 0); the mode m = (-1, 0) is its mirror and is implied.
    Shape (2, N, N//2), complex128.
    """
    u = np.zeros((2, N, N // 2), dtype=np.complex128)
    u[1, 0, 1] = -0.5j
    return u


def config_ns2d_circle(N: int = 64, Nb: int = 202, dt: float = 1e-3, T: float = 10.0,
                       precision: str = "fp64") -> Problem:
    """Circle of radius L/4 at the box centre in the sine flow (Sec. 5.2.1).

    N = 64, N_b = 202 (h_b close to L/N), dt = 1e-3, K = 1, rho = 1, mu = 0.01, and
    the boundary released in u_0 = (0, sin(2 pi x/L)); T = 10 is long enough for the
    boundary to return to a circle.
    """
    X0 = ellipse(Nb, 0.25 * L_BOX, 0.25 * L_BOX, (0.5 * L_BOX, 0.5 * L_BOX))
    tol = 1e-12 if precision == "fp64" else 1e-6
    nsteps = int(round(T / dt))
    return Problem(f"ns2d_circle_N{N}_Nb{Nb}_{precision}", 2, N, Nb, 0.01, 1.0, dt, nsteps, tol,
                   precision, "curve", X0, 1.0, extra={"u0": sine_velocity_half(N), "T": T})


def channel_targets(N: int) -> np.ndarray:
    """Target points of the two channel walls (Sec. 5.2.2): X~_i = (i h, L/4) and
    X~_{i+N} = (i h, 3L/4), i = 0..N-1, h = L/N; shape (2, 2N)."""
    h = L_BOX / N
    x = h * np.arange(N, dtype=np.float64)
    lo = np.stack([x, np.full(N, 0.25 * L_BOX)])
    hi = np.stack([x, np.full(N, 0.75 * L_BOX)])
    return np.concatenate([lo, hi], axis=1)


def config_poiseuille(N: int = 8, K: float = 1.0e4, T: float = 3.0, dt: float | None = None,
                      precision: str = "fp64") -> Problem:
    """Navier-Stokes flow in a channel with target-point walls (Sec. 5.2.2).

    L = 1, mu = 0.1, rho = 1, body force f0 = 100 along x, walls at y = L/4 and 3L/4
    (D = L/2) with N_b = 2N markers started on their targets, fluid at rest.
    The paper states neither the target stiffness K nor dt: K = 1e4 and
    dt = 1e-3 * 8/N (dt proportional to h) keep the explicit spring stable, and
    T = 3 is about twelve decay times of the slowest channel mode
    (rate mu (pi/D)^2 / rho = 3.95), so the flux is steady to about 1e-5.
    """
    if dt is None:
        dt = 1e-3 * 8.0 / N
    Xt = channel_targets(N)
    h = L_BOX / N
    tol = 1e-12 if precision == "fp64" else 1e-6
    nsteps = int(round(T / dt))
    return Problem(f"poiseuille_N{N}_{precision}", 2, N, 2 * N, 0.1, 1.0, dt, nsteps, tol,
                   precision, "target", Xt.copy(), K,
                   extra={"Xtarget": Xt, "omega": h, "fbody": (100.0, 0.0), "band": (0.25, 0.75),
                          "D": 0.5 * L_BOX, "f0": 100.0, "T": T})


# ---------------------------------------------------------------------------
# Three-dimensional sphere problems of Secs. 6.2.3 (elastic) and 6.2.4 (surface tension)
# ---------------------------------------------------------------------------

def sine_velocity_half_3d(N: int) -> np.ndarray:
    """Initial velocity u_0 = (sin(2 pi z/L), 0, sin(2 pi y/L)) in the half-spectrum layout.

    Both sines live on the plane m_x = 0, which stores every (m_y, m_z): the x component
    holds -i/2 at m_z = 1 and +i/2 at m_z = -1, the z component the same along m_y.
    Shape (3, N, N, N//2), complex128, indexed [component, iz, iy, ix].
    """
    u = np.zeros((3, N, N, N // 2), dtype=np.complex128)
    u[0, 1, 0, 0], u[0, N - 1, 0, 0] = -0.5j, 0.5j
    u[2, 0, 1, 0], u[2, 0, N - 1, 0] = -0.5j, 0.5j
    return u


def config_ns3d_sphere(model: str = "elastic", level: int = 4, N: int = 32, dt: float = 1e-3,
                       T: float = 1.0, precision: str = "fp64") -> Problem:
    """Sphere of radius L/3 at the box centre in the sine flow u_0 = (sin 2 pi z, 0, sin 2 pi y).

    model "elastic": cot-weight springs with sigma = 1 from the initial sphere (Sec. 6.2.3);
    model "tension": surface tension gamma = 1 (Sec. 6.2.4). L = 1, rho = 1, mu = 0.01,
    N = 32 with four refinements of the icosahedron (M = 2562) so that the Lagrangian
    meshwidth matches the Fourier resolution, dt = 1e-3, T = 1.
    """
    X0, tri = icosphere(level, L_BOX / 3.0, (0.5, 0.5, 0.5))
    tol = 1e-12 if precision == "fp64" else 1e-6
    nsteps = int(round(T / dt))
    force = "mesh" if model == "elastic" else "tension"
    return Problem(f"ns3d_sphere_{model}_L{level}_N{N}_{precision}", 3, N, X0.shape[1], 0.01, 1.0, dt,
                   nsteps, tol, precision, force, X0.copy(), 1.0, tri=tri, Xref=X0.copy(),
                   extra={"u0": sine_velocity_half_3d(N), "T": T, "level": level})
