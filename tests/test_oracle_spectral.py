"""Pins of the oracle's spectral functions against what the paper and mathematics fix.

Every check compares the oracle with something other than itself: brute-force
loops, a library FFT on points that sit on a grid, closed forms, or identities
the paper proves.
"""
import math

import numpy as np
import pytest

from oracle import spectral as sp
from paper_2302_08694_gb300 import workloads as wl

TWO_PI = 2 * math.pi


def _hermitian_full(rng, nc, N, d):
    shape = (nc,) + (N,) * (d - 1) + (N // 2,)
    H = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return sp.half_to_full(H, N, d)


# P1: direct separable sums vs plain loops --------------------------------------------------

@pytest.mark.parametrize("d,N,M", [(2, 6, 7), (3, 4, 5), (2, 5, 4), (3, 6, 3)])
def test_spread_interp_match_brute_force(d, N, M):
    rng = np.random.default_rng(10 + d + N)
    X = rng.uniform(-0.3, 1.7, (d, M))
    c = rng.standard_normal((d, M))
    A = sp.spread_direct(X, c, N, chunk=3)
    B = sp.spread_brute(X, c, N)
    assert np.max(np.abs(A - B)) <= 1e-14 * max(1.0, np.max(np.abs(B)))
    Fu = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
    U1 = sp.interp_direct_complex(Fu, X, N, chunk=2)
    U2 = sp.interp_brute(Fu, X, N)
    assert np.max(np.abs(U1 - U2)) <= 1e-13 * max(1.0, np.max(np.abs(U2)))


def test_box_length_scaling():
    # The sums with box L and positions L*X equal L^-d times the unit-box sums.
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (2, 9))
    c = rng.standard_normal((2, 9))
    A = sp.spread_direct(X, c, 8, L=1.0)
    B = sp.spread_direct(2.5 * X, c, 8, L=2.5)
    assert np.allclose(B, A / 2.5 ** 2, rtol=0, atol=1e-14)


# P2: points on the grid reduce type-1 to the DFT and type-2 to the inverse DFT ------------

@pytest.mark.parametrize("d,N", [(2, 8), (3, 6), (2, 12)])
def test_on_grid_points_are_dft(d, N):
    rng = np.random.default_rng(5)
    L = 1.0
    h = L / N
    grid = np.meshgrid(*([np.arange(N) * h] * d), indexing="ij")  # grid[a][i0, i1, ...]
    # point order: array index (iz, iy, ix); X[0] = x varies along the last index
    X = np.stack([grid[d - 1 - a].ravel() for a in range(d)])
    g = rng.standard_normal((N,) * d)  # field sampled on the grid, g[iz, iy, ix]
    # X[a][j] = h * (index along axis a); the array index of point j along axis a:
    ia = [np.rint(X[a] / h).astype(int) for a in range(d)]
    vals = g[tuple(ia[::-1])]
    c = (h ** d) * vals[None, :]
    fhat = sp.spread_direct(X, c, N)
    ref = np.fft.fftn(g) / N ** d
    ref = sp.zero_nyquist(ref[None], N, d)
    assert np.max(np.abs(fhat - ref)) <= 1e-14
    # type-2 on the grid: u(x_n) = N^d * ifftn(u-hat)
    Fu = _hermitian_full(rng, 1, N, d)
    U = sp.interp_direct(Fu, X, N)
    grid_u = (np.fft.ifftn(Fu[0]) * N ** d).real
    assert np.max(np.abs(U[0] - grid_u[tuple(ia[::-1])])) <= 1e-12


# P13: the library FFT the oracle's dealiasing uses agrees with a direct DFT ---------------

@pytest.mark.parametrize("n", [6, 8, 9, 12, 16, 18, 24])
def test_numpy_fft_is_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    Wm = np.exp(-2j * np.pi * np.outer(j, j) / n)
    assert np.allclose(np.fft.fft(x), Wm @ x, rtol=0, atol=1e-12)
    assert np.allclose(np.fft.ifft(x) * n, np.conj(Wm) @ x, rtol=0, atol=1e-12)


# Half-spectrum layout ----------------------------------------------------------------------

@pytest.mark.parametrize("d,N", [(2, 8), (3, 6), (3, 8)])
def test_half_spectrum_roundtrip_and_realness(d, N):
    rng = np.random.default_rng(7)
    shape = (2,) + (N,) * (d - 1) + (N // 2,)
    H = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Fu = sp.half_to_full(H, N, d)
    assert sp.is_hermitian(Fu, N, d)
    # the interpolated field of the full spectrum is real at arbitrary points
    X = rng.uniform(0, 1, (d, 11))
    Uc = sp.interp_direct_complex(Fu, X, N)
    assert np.max(np.abs(Uc.imag)) <= 1e-12 * np.max(np.abs(Uc))
    # equals the explicit half sum: Re(sum_{mx=0} H e) + 2 Re(sum_{mx>0} H e), Nyquist dropped
    m = sp.mode_ints(N)
    U = np.zeros((2, X.shape[1]))
    for idx in np.ndindex(*shape[1:]):
        mv = [idx[-1]] + [m[idx[-2 - a]] for a in range(d - 1)]  # (mx, my, mz)
        if any(v == -N // 2 for v in mv):
            continue
        ph = sum(TWO_PI * mv[a] * X[a] for a in range(d))
        w = 1.0 if mv[0] == 0 else 2.0
        for q in range(2):
            U[q] += w * np.real(H[(q,) + idx] * np.exp(1j * ph))
    assert np.max(np.abs(Uc.real - U)) <= 1e-12 * np.max(np.abs(U))
    # and a Hermitian spectrum survives full -> half -> full
    assert np.allclose(sp.half_to_full(sp.full_to_half(Fu, N), N, d), Fu, atol=1e-15)


# P11: spread then interp of a unit source is the periodised sinc kernel ---------------------

@pytest.mark.parametrize("d,N", [(1 + 1, 8), (3, 6), (2, 10)])
def test_kernel_identity(d, N):
    """With the Nyquist mode dropped, K_N for even N is the symmetric set of N-1
    modes, and spread-then-interp of a unit source gives prod_a delta_{L,N-1}(dx_a),
    delta_{L,n}(x) = sin(n pi x/L)/(L sin(pi x/L)) (Eq. FSIB_kern_odd)."""
    rng = np.random.default_rng(11)
    L = 1.0
    x1 = rng.uniform(0, 1, (d, 1))
    x2 = rng.uniform(0, 1, (d, 5))
    fhat = sp.spread_direct(x1, np.ones((1, 1)), N, L)
    U = sp.interp_direct(fhat, x2, N, L)[0]
    n = N - 1
    ref = np.ones(5)
    for a in range(d):
        dx = x2[a] - x1[a, 0]
        ref *= np.sin(n * np.pi * dx / L) / (L * np.sin(np.pi * dx / L))
    assert np.allclose(U, ref, rtol=1e-12, atol=1e-12)
    # sum of squares on the grid (Eq. sum_square_FSIB, 1D factor): sum_j delta(x - j h)^2 h = delta(0)
    h = L / n
    j = np.arange(n)
    x = 0.37
    dlt = np.sin(n * np.pi * (x - j * h) / L) / (L * np.sin(np.pi * (x - j * h) / L))
    assert abs(np.sum(dlt ** 2) * h - n / L) <= 1e-11


# P3: duality of spread and interp ----------------------------------------------------------

@pytest.mark.parametrize("d,N,M", [(2, 8, 13), (3, 6, 9)])
def test_duality(d, N, M):
    """L^d sum_k f-hat(k) . conj(u-hat(k)) = sum_j omega_j F_j . U_j (Eq. pote_energ_derivative)."""
    rng = np.random.default_rng(17)
    L = 1.3
    X = rng.uniform(0, L, (d, M))
    c = rng.standard_normal((d, M))
    Fu = _hermitian_full(rng, d, N, d)
    fhat = sp.spread_direct(X, c, N, L)
    U = sp.interp_direct(Fu, X, N, L)
    lhs = L ** d * np.sum(fhat * np.conj(Fu))
    rhs = np.sum(c * U)
    assert abs(lhs.imag) <= 1e-12 * abs(rhs)
    assert abs(lhs.real - rhs) <= 1e-12 * np.sum(np.abs(c) * np.abs(U))


# P4 / P9: Stokeslet -------------------------------------------------------------------------

def test_stokes_sinusoid_closed_form():
    """Body force f = (0, sin(2 pi x/L)) on grid points: u = (0, L^2 sin(2 pi x/L)/(4 pi^2 mu)) (Eq. stokeslet)."""
    N, mu, L = 8, 0.7, 1.0
    h = L / N
    gx, gy = np.meshgrid(np.arange(N) * h, np.arange(N) * h, indexing="xy")
    X = np.stack([gx.ravel(), gy.ravel()])
    c = np.zeros_like(X)
    c[1] = h * h * np.sin(TWO_PI * X[0] / L)
    fhat = sp.spread_direct(X, c, N, L)
    uhat = sp.stokeslet(fhat, N, mu, L)
    rng = np.random.default_rng(1)
    Y = rng.uniform(0, 1, (2, 20))
    U = sp.interp_direct(uhat, Y, N, L)
    assert np.max(np.abs(U[0])) <= 1e-14
    ref = L ** 2 * np.sin(TWO_PI * Y[0] / L) / (4 * np.pi ** 2 * mu)
    assert np.max(np.abs(U[1] - ref)) <= 1e-14


@pytest.mark.parametrize("d,N", [(2, 8), (3, 6)])
def test_stokeslet_divergence_free_and_solves_stokes(d, N):
    rng = np.random.default_rng(2)
    mu = 0.3
    F = _hermitian_full(rng, d, N, d)
    u = sp.stokeslet(F, N, mu)
    assert sp.max_divergence(u, N) <= 1e-14  # a few ulps of rounding
    # mu |k|^2 u = P f on k != 0: the Stokes equations with the pressure removed
    k2 = sp.ksq(N, d)
    Pf = sp.leray(F, N)
    nz = k2 > 0
    for a in range(d):
        assert np.allclose((mu * k2 * u[a])[nz], sp.zero_nyquist(Pf, N, d)[a][nz], atol=1e-13)
    assert np.all(u[(slice(None),) + (0,) * d] == 0)


# P12 / P7: dealiased nonlinear term ---------------------------------------------------------

@pytest.mark.parametrize("d,N", [(2, 6), (2, 8), (3, 4)])
def test_dealiasing_exact(d, N):
    """The three-halves rule reproduces the direct convolution over K_N exactly (Sec. 3.1)."""
    rng = np.random.default_rng(23)
    u = sp.leray(_hermitian_full(rng, d, N, d), N)
    s1 = sp.nonlinear(u, N)
    s2 = sp.nonlinear_direct(u, N)
    assert np.max(np.abs(s1 - s2)) <= 1e-12 * np.max(np.abs(s2))
    # the smallest alias-free grid is 3N/2 - 2; one point less aliases
    s4 = sp.nonlinear(u, N, Nt=3 * N // 2 - 2)
    assert np.max(np.abs(s4 - s2)) <= 1e-12 * np.max(np.abs(s2))
    if 3 * N // 2 - 3 >= N:
        s3 = sp.nonlinear(u, N, Nt=3 * N // 2 - 3)
        assert np.max(np.abs(s3 - s2)) > 1e-6 * np.max(np.abs(s2))


@pytest.mark.parametrize("d,N", [(2, 8), (3, 6)])
def test_nonlinear_energy_neutral_and_zero_mean(d, N):
    """sum_k s-hat(k) . conj(u-hat(k)) = 0 and s-hat(0) = 0 for divergence-free u (Secs. 4.3, 4.4)."""
    rng = np.random.default_rng(29)
    u = sp.leray(_hermitian_full(rng, d, N, d), N)
    s = sp.nonlinear(u, N)
    tot = np.sum(s * np.conj(u))
    assert abs(tot) <= 1e-12 * np.sum(np.abs(s) * np.abs(u))
    assert np.max(np.abs(s[(slice(None),) + (0,) * d])) <= 1e-13 * np.max(np.abs(s))


def test_vhat_is_divergence_free():
    rng = np.random.default_rng(31)
    N, d = 6, 3
    u = sp.leray(_hermitian_full(rng, d, N, d), N)
    f = _hermitian_full(rng, d, N, d)
    V = sp.vhat(f, u, N, rho=1.7)
    assert sp.max_divergence(V, N) <= 1e-14


def test_shear_flow_follows_be_cn_recurrence():
    """u = (0, a sin(2 pi x)) makes u . grad u = 0, so the substeps reduce to
    a_half = (dt/2 f/rho + a)/(1 + lam/2) and a1 = (dt f/rho + (1 - lam/2) a)/(1 + lam/2),
    lam = mu dt |k|^2/rho (Eqs. spatial_2, spatial_3)."""
    N, d = 8, 2
    mu, rho, dt = 0.05, 1.3, 0.01
    a, fa = 0.8, 2.0
    u = np.zeros((2, N, N), dtype=complex)
    f = np.zeros((2, N, N), dtype=complex)
    # sin(2 pi x) = (e^{i 2pi x} - e^{-i 2pi x})/(2i): modes m_x = +1, -1 at (iy = 0, ix = 1, N-1)
    for coef, arr in ((a, u), (fa, f)):
        arr[1, 0, 1] = coef / 2j
        arr[1, 0, N - 1] = -coef / 2j
    uh, u1 = sp.ns_substeps(f, u, N, mu, rho, dt)
    lam = mu * dt * (TWO_PI) ** 2 / rho
    ah = (0.5 * dt * fa / rho + a) / (1 + lam / 2)
    a1 = (dt * fa / rho + (1 - lam / 2) * a) / (1 + lam / 2)
    assert abs(uh[1, 0, 1] - ah / 2j) <= 1e-15
    assert abs(u1[1, 0, 1] - a1 / 2j) <= 1e-15
    assert np.max(np.abs(u1[0])) == 0.0


# P15: spectral accuracy of the trapezoid spread on a closed curve ---------------------------

def test_trapezoid_spread_converges_exponentially():
    N = 8
    c0 = np.array([0.5, 0.5])

    def fh(M):
        X = wl.ellipse(M, 0.2, 0.2, c0)
        th = 2 * np.pi * np.arange(M) / M
        F = np.stack([np.cos(th) + 0.3 * np.sin(2 * th), np.sin(th)])
        return sp.spread_direct(X, (2 * np.pi / M) * F, N)

    ref = fh(512)
    errs = [np.max(np.abs(fh(M) - ref)) for M in (8, 16, 32)]
    assert errs[1] < 1e-2 * errs[0]
    assert errs[2] < 1e-12


def test_spread_at_modes_matches_full_sum():
    rng = np.random.default_rng(41)
    X = rng.uniform(0, 1, (3, 17))
    c = rng.standard_normal((3, 17))
    N = 6
    F = sp.spread_direct(X, c, N)
    m = sp.mode_ints(N)
    idx = rng.integers(0, N, (9, 3))
    modes = np.stack([m[idx[:, 0]], m[idx[:, 1]], m[idx[:, 2]]], axis=1)  # (mx, my, mz)
    S = sp.spread_at_modes(X, c, modes)
    for q in range(9):
        if any(v == -N // 2 for v in modes[q]):
            continue
        assert np.allclose(S[:, q], F[:, idx[q, 2], idx[q, 1], idx[q, 0]], atol=1e-14)
