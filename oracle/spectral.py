"""Spectral part of the oracle: mode set, direct non-uniform sums, fluid solve.

Full-spectrum arrays have shape (ncomp, N, N) in 2D and (ncomp, N, N, N) in 3D,
indexed [component, (iz,) iy, ix] with every axis in FFT order (index i holds
integer mode m = i for i < N/2, m = i - N otherwise). Component 0 is x. The
wavenumber of an entry is k = 2*pi*m/L per axis (physical, Sec. 2).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# Mode set K_N (Eq. kNh)
# ---------------------------------------------------------------------------

def mode_ints(N: int) -> np.ndarray:
    """Integer modes of one axis in FFT order: even N gives -N/2..N/2-1 (Eq. kNh)."""
    i = np.arange(N, dtype=np.int64)
    return np.where(i < (N + 1) // 2, i, i - N)


def nyquist_mask(N: int, d: int) -> np.ndarray:
    """Boolean array (N,)*d, True where some axis holds the unpaired mode -N/2.

    Eq. kNh keeps m = -N/2 but not +N/2 for even N. The oracle zeroes those
    modes so that the kept set is symmetric (the reading used throughout).
    """
    m = mode_ints(N)
    ny = (m == -N // 2) if N % 2 == 0 else np.zeros(N, dtype=bool)
    grids = np.meshgrid(*([ny] * d), indexing="ij")
    out = np.zeros((N,) * d, dtype=bool)
    for g in grids:
        out |= g
    return out


def wavevectors(N: int, d: int, L: float = 1.0):
    """List [k_x, k_y, (k_z)] broadcast to shape (N,)*d; k_x varies along the last axis."""
    k1 = TWO_PI / L * mode_ints(N).astype(np.float64)
    ks = []
    for a in range(d):  # a = 0 is x = last array axis
        shape = [1] * d
        shape[d - 1 - a] = N
        ks.append(np.broadcast_to(k1.reshape(shape), (N,) * d))
    return ks


def ksq(N: int, d: int, L: float = 1.0) -> np.ndarray:
    ks = wavevectors(N, d, L)
    return sum(k * k for k in ks)


def zero_nyquist(F: np.ndarray, N: int, d: int) -> np.ndarray:
    G = F.copy()
    G[..., nyquist_mask(N, d)] = 0.0
    return G


# ---------------------------------------------------------------------------
# Half-spectrum layout of the library (m_x >= 0 only)
# ---------------------------------------------------------------------------

def half_to_full(H: np.ndarray, N: int, d: int) -> np.ndarray:
    """Full spectrum represented by a half-spectrum array.

    H has shape (ncomp, (N,) N, N/2): all m_y (m_z) in FFT order and m_x = 0..N/2-1.
    Represented spectrum: u(m) = H(m) for m_x > 0, u(m) = conj(H(-m)) for m_x < 0,
    and on the plane m_x = 0 the Hermitian part (H(m) + conj(H(-m)))/2.
    Nyquist modes are zero. This is the spectrum of a real field.
    """
    nc = H.shape[0]
    Fu = np.zeros((nc,) + (N,) * d, dtype=np.complex128)
    h = N // 2
    Fu[..., :h] = H
    neg = (-np.arange(N)) % N  # index of -m along one axis
    # m_x < 0: ix in (h, N) holds mode ix - N; its mirror -m has m_x = N - ix in (0, h)
    idx_other = np.ix_(*([neg] * (d - 1)))
    for ix in range(h + 1, N):
        src = H[(slice(None),) + (Ellipsis,) + (N - ix,)]
        Fu[..., ix] = np.conj(src[(slice(None),) + idx_other])
    plane0 = H[..., 0]
    Fu[..., 0] = 0.5 * (plane0 + np.conj(plane0[(slice(None),) + idx_other]))
    return zero_nyquist(Fu, N, d)


def full_to_half(F: np.ndarray, N: int) -> np.ndarray:
    """Half-spectrum view of a Hermitian full spectrum (modes m_x = 0..N/2-1)."""
    return np.ascontiguousarray(F[..., : N // 2])


def is_hermitian(F: np.ndarray, N: int, d: int, rtol=1e-13) -> bool:
    neg = (-np.arange(N)) % N
    G = np.conj(F[(slice(None),) + np.ix_(*([neg] * d))])
    return np.max(np.abs(F - G)) <= rtol * max(np.max(np.abs(F)), 1e-300)


# ---------------------------------------------------------------------------
# Direct type-1 / type-2 sums (Eqs. force_spreading_quad, velo_intp_fini)
# ---------------------------------------------------------------------------

def _phase(X_a: np.ndarray, N: int, L: float, sign: float) -> np.ndarray:
    """E[j, i] = exp(sign * i * k(i) * X_a[j]) for one axis, k in FFT order."""
    k = TWO_PI / L * mode_ints(N).astype(np.float64)
    return np.exp(sign * 1j * np.outer(X_a, k))


def spread_direct(X: np.ndarray, c: np.ndarray, N: int, L: float = 1.0,
                  chunk: int = 2048) -> np.ndarray:
    """f-hat(k) = L^-d sum_j c_j exp(-i k . X_j), k in K_N (Eq. force_spreading_quad).

    c = omega_j F_j with shape (ncomp, M). Separable evaluation: the phase is a
    product over axes; the sum over j is a matrix product per chunk of points.
    Nyquist modes are zeroed. Returns the full spectrum (ncomp, (N,)*d).
    """
    d, M = X.shape
    nc = c.shape[0]
    out = np.zeros((nc,) + (N,) * d, dtype=np.complex128)
    flat = out.reshape(nc, N, N ** (d - 1))
    for j0 in range(0, M, chunk):
        j1 = min(M, j0 + chunk)
        Ex = _phase(X[0, j0:j1], N, L, -1.0)
        Ey = _phase(X[1, j0:j1], N, L, -1.0)
        if d == 2:
            # out[c, iy, ix] = sum_j c[c,j] Ey[j,iy] Ex[j,ix]
            B = (c[:, j0:j1, None] * Ey[None, :, :])  # (nc, mc, N)
            flat += np.einsum("cjy,jx->cyx", B, Ex).reshape(nc, N, N)
        else:
            Ez = _phase(X[2, j0:j1], N, L, -1.0)
            A = (Ey[:, :, None] * Ex[:, None, :]).reshape(j1 - j0, N * N)
            B = (c[:, j0:j1, None] * Ez[None, :, :])  # (nc, mc, N)
            B = np.transpose(B, (0, 2, 1)).reshape(nc * N, j1 - j0)
            flat += (B @ A).reshape(nc, N, N * N)
    out *= L ** (-d)
    return zero_nyquist(out, N, d)


def interp_direct_complex(Fu: np.ndarray, X: np.ndarray, N: int, L: float = 1.0,
                          chunk: int = 2048) -> np.ndarray:
    """U_j = sum_{k in K_N} u-hat(k) exp(i k . X_j) (Eq. velo_intp_fini), complex result."""
    d, M = X.shape
    nc = Fu.shape[0]
    U = np.zeros((nc, M), dtype=np.complex128)
    for j0 in range(0, M, chunk):
        j1 = min(M, j0 + chunk)
        Ex = _phase(X[0, j0:j1], N, L, 1.0)
        Ey = _phase(X[1, j0:j1], N, L, 1.0)
        if d == 2:
            T = np.einsum("cyx,jx->cyj", Fu, Ex)
            U[:, j0:j1] = np.einsum("cyj,jy->cj", T, Ey)
        else:
            Ez = _phase(X[2, j0:j1], N, L, 1.0)
            A = (Ey[:, :, None] * Ex[:, None, :]).reshape(j1 - j0, N * N)
            T = Fu.reshape(nc * N, N * N) @ A.T  # (nc*N, mc)
            T = T.reshape(nc, N, j1 - j0)
            U[:, j0:j1] = np.einsum("czj,jz->cj", T, Ez)
    return U


def interp_direct(Fu: np.ndarray, X: np.ndarray, N: int, L: float = 1.0,
                  chunk: int = 2048, imag_rtol: float = 1e-14) -> np.ndarray:
    """Real velocity at the points. The imaginary part is checked, not dropped silently."""
    Uc = interp_direct_complex(Fu, X, N, L, chunk)
    scale = max(float(np.max(np.abs(Uc))) if Uc.size else 0.0, 1e-300)
    im = float(np.max(np.abs(Uc.imag))) if Uc.size else 0.0
    if im > imag_rtol * scale and im > 1e-280:
        raise ValueError(f"interp: imaginary part {im:.3e} vs scale {scale:.3e}; "
                         "u-hat is not the spectrum of a real field")
    return np.ascontiguousarray(Uc.real)


def spread_brute(X, c, N, L=1.0):
    """Same sum as spread_direct, by plain loops over points and modes (tiny inputs)."""
    d, M = X.shape
    nc = c.shape[0]
    m = mode_ints(N)
    out = np.zeros((nc,) + (N,) * d, dtype=np.complex128)
    for idx in np.ndindex(*((N,) * d)):
        mv = [m[idx[d - 1 - a]] for a in range(d)]  # a = 0 is x (last index)
        if N % 2 == 0 and any(v == -N // 2 for v in mv):
            continue
        for j in range(M):
            ph = sum(TWO_PI / L * mv[a] * X[a, j] for a in range(d))
            e = complex(math.cos(ph), -math.sin(ph))
            for q in range(nc):
                out[(q,) + idx] += c[q, j] * e
    return out / L ** d


def interp_brute(Fu, X, N, L=1.0):
    d, M = X.shape
    nc = Fu.shape[0]
    m = mode_ints(N)
    U = np.zeros((nc, M), dtype=np.complex128)
    for j in range(M):
        for idx in np.ndindex(*((N,) * d)):
            mv = [m[idx[d - 1 - a]] for a in range(d)]
            ph = sum(TWO_PI / L * mv[a] * X[a, j] for a in range(d))
            e = complex(math.cos(ph), math.sin(ph))
            for q in range(nc):
                U[q, j] += Fu[(q,) + idx] * e
    return U


# ---------------------------------------------------------------------------
# Fluid solve
# ---------------------------------------------------------------------------

def stokeslet(fhat: np.ndarray, N: int, mu: float, L: float = 1.0) -> np.ndarray:
    """u-hat = mu^-1 (I/|k|^2 - k k^T/|k|^4) f-hat, u-hat(0) = 0 (Eq. stokeslet).

    The k = 0 mode has no solution unless the net force vanishes (Eq.
    force_vanish); the oracle sets it to zero.
    """
    d = fhat.shape[0]
    ks = wavevectors(N, d, L)
    k2 = sum(k * k for k in ks)
    zero = k2 == 0.0
    k2s = np.where(zero, 1.0, k2)
    kf = sum(ks[a] * fhat[a] for a in range(d))
    u = np.empty_like(fhat)
    for a in range(d):
        u[a] = (fhat[a] / k2s - ks[a] * kf / (k2s * k2s)) / mu
        u[a][zero] = 0.0
    return zero_nyquist(u, N, d)


def leray(P: np.ndarray, N: int, L: float = 1.0) -> np.ndarray:
    """Q = P - k (k . P)/|k|^2 with |k|^2 := 1 at k = 0 (Algorithm 2)."""
    d = P.shape[0]
    ks = wavevectors(N, d, L)
    k2 = sum(k * k for k in ks)
    k2 = np.where(k2 == 0.0, 1.0, k2)
    kP = sum(ks[a] * P[a] for a in range(d))
    return np.stack([P[a] - ks[a] * kP / k2 for a in range(d)])


def _pad_index(N: int, Nt: int) -> np.ndarray:
    """Position of each length-N FFT-order mode inside a length-Nt FFT-order array."""
    return mode_ints(N) % Nt


def nonlinear(uhat: np.ndarray, N: int, L: float = 1.0, Nt: int | None = None) -> np.ndarray:
    """s-hat = T_N H((H^-1 u-hat) . (H^-1 i k u-hat)) by the three-halves rule (Eq. nonlinear_kspace).

    Steps in the order of Sec. 3.1: form i k_b u-hat_a; zero-pad u-hat and the
    gradient to N~ per axis (centred padding); inverse transform to the N~^d
    grid; s_a = sum_b u_b d_b u_a (convective form); forward transform; keep
    K_N; zero the Nyquist modes. N~ defaults to 3N/2. With the Nyquist mode
    dropped the kept modes of an axis are |m| <= K = N/2 - 1, products hold
    |m| <= 2K, and an alias m -+ N~ of a product mode lands in the kept set
    only if N~ <= 3K; so any N~ >= 3N/2 - 2 is alias-free and 3N/2 has a
    margin of two.
    """
    d = uhat.shape[0]
    if Nt is None:
        Nt = 3 * N // 2
    ks = wavevectors(N, d, L)
    idx = _pad_index(N, Nt)
    sel = np.ix_(*([idx] * d))

    def to_grid(v):
        P = np.zeros((Nt,) * d, dtype=np.complex128)
        P[sel] = v
        # grid value g(x_n) = sum_k v(k) exp(i k . x_n), x_n = L n / Nt
        return np.fft.ifftn(P) * Nt ** d

    u = [to_grid(uhat[a]).real for a in range(d)]
    s = []
    for a in range(d):
        sa = np.zeros((Nt,) * d)
        for b in range(d):
            sa += u[b] * to_grid(1j * ks[b] * uhat[a]).real
        s.append(sa)
    out = np.empty_like(uhat)
    for a in range(d):
        S = np.fft.fftn(s[a]) / Nt ** d
        out[a] = S[sel]
    return zero_nyquist(out, N, d)


def nonlinear_direct(uhat: np.ndarray, N: int, L: float = 1.0) -> np.ndarray:
    """s-hat(k) = sum_{k1} (u-hat(k-k1) . i k1) u-hat(k1), k, k1, k-k1 in K_N (convolution form, Sec. 5.2.2)."""
    d = uhat.shape[0]
    m = mode_ints(N)
    kept = [v for v in m if not (N % 2 == 0 and v == -N // 2)]
    pos = {int(v): int(i) for i, v in enumerate(m)}
    out = np.zeros_like(uhat)
    for idx in np.ndindex(*((N,) * d)):
        mv = [int(m[idx[d - 1 - a]]) for a in range(d)]
        if any(v not in kept for v in mv):
            continue
        acc = np.zeros(d, dtype=np.complex128)
        for k1 in np.ndindex(*((len(kept),) * d)):
            m1 = [kept[k1[a]] for a in range(d)]
            m2 = [mv[a] - m1[a] for a in range(d)]
            if any(v not in kept for v in m2):
                continue
            i1 = tuple(pos[m1[d - 1 - a]] for a in range(d))
            i2 = tuple(pos[m2[d - 1 - a]] for a in range(d))
            u1 = uhat[(slice(None),) + i1]
            u2 = uhat[(slice(None),) + i2]
            dot = sum(u2[b] * 1j * TWO_PI / L * m1[b] for b in range(d))
            acc += dot * u1
        out[(slice(None),) + idx] = acc
    return out


def vhat(fhat: np.ndarray, uhat: np.ndarray, N: int, rho: float, L: float = 1.0,
         Nt: int | None = None) -> np.ndarray:
    """V-hat(f-hat, u-hat) = P_k (f-hat/rho - s-hat(u-hat)) (Eq. fourier_spectral_sol, Algorithm 2)."""
    P = fhat / rho - nonlinear(uhat, N, L, Nt)
    d = fhat.shape[0]
    return zero_nyquist(leray(P, N, L), N, d)


def ns_substeps(fhat: np.ndarray, uhat: np.ndarray, N: int, mu: float, rho: float,
                dt: float, L: float = 1.0, Nt: int | None = None):
    """Backward-Euler half step and Crank-Nicolson full step (Eqs. spatial_2, spatial_3; Algorithm 1).

    u-hat^{m+1/2} = (dt/2 V(f, u^m) + u^m) / (1 + mu dt |k|^2 / (2 rho))
    u-hat^{m+1}   = (dt V(f, u^{m+1/2}) + (1 - mu dt |k|^2/(2 rho)) u^m) / (1 + mu dt |k|^2/(2 rho))
    """
    d = fhat.shape[0]
    lam = mu * dt * ksq(N, d, L) / rho
    den = 1.0 + 0.5 * lam
    uh = (0.5 * dt * vhat(fhat, uhat, N, rho, L, Nt) + uhat) / den
    u1 = (dt * vhat(fhat, uh, N, rho, L, Nt) + (1.0 - 0.5 * lam) * uhat) / den
    return zero_nyquist(uh, N, d), zero_nyquist(u1, N, d)


# ---------------------------------------------------------------------------
# Spectral diagnostics (Sec. 4)
# ---------------------------------------------------------------------------

def pressure(fhat: np.ndarray, uhat, N: int, rho: float, L: float = 1.0,
             Nt: int | None = None) -> np.ndarray:
    """Pressure p-hat = -i k.(f-hat - rho s-hat(u-hat)) / |k|^2 with p-hat(0) = 0
    (Eq. pressure_poisson_k; the constant is free and chosen so that p has mean zero).
    uhat None drops the nonlinear term (Stokes). Returns one full-spectrum component."""
    d = fhat.shape[0]
    P = fhat if uhat is None else fhat - rho * nonlinear(uhat, N, L, Nt)
    ks = wavevectors(N, d, L)
    kP = sum(ks[a] * P[a] for a in range(d))
    k2 = ksq(N, d, L)
    p = np.where(k2 > 0, -1j * kP / np.where(k2 > 0, k2, 1.0), 0.0)
    return zero_nyquist(p[None], N, d)[0]


def band_flux(uhat: np.ndarray, N: int, comp: int, axis: int, y0: float, y1: float,
              L: float = 1.0) -> float:
    """Flux of velocity component `comp` through the band y0 <= x_axis <= y1.

    Phi = int_{y0}^{y1} ubar(y) dy, where ubar is u_comp averaged over the other
    axes (the channel flux of Eq. poiseuille_flux for a laminar flow). Only the
    modes m e_axis survive the average: ubar(y) = sum_m u-hat(m e_axis) e^{i k_m y}.
    """
    d = uhat.shape[0]
    m = mode_ints(N).astype(np.float64)
    k = TWO_PI / L * m
    idx = [0] * d
    acc = 0.0 + 0.0j
    for i in range(N):
        idx[d - 1 - axis] = i
        if k[i] == 0.0:
            I = y1 - y0
        else:
            I = (np.exp(1j * k[i] * y1) - np.exp(1j * k[i] * y0)) / (1j * k[i])
        acc += uhat[(comp,) + tuple(idx)] * I
    return float(acc.real)


def kinetic_energy(uhat: np.ndarray, N: int, rho: float, L: float = 1.0) -> float:
    """E_K = (1/2) rho L^d sum_k u-hat(k) . conj(u-hat(k)) (Sec. 4.4)."""
    d = uhat.shape[0]
    return float(0.5 * rho * L ** d * np.sum(np.abs(uhat) ** 2))


def dissipation(uhat: np.ndarray, N: int, mu: float, L: float = 1.0) -> float:
    """mu L^d sum_k |k|^2 |u-hat(k)|^2, the viscous dissipation rate (Sec. 4.4)."""
    d = uhat.shape[0]
    return float(mu * L ** d * np.sum(ksq(N, d, L) * np.sum(np.abs(uhat) ** 2, axis=0)))


def max_divergence(uhat: np.ndarray, N: int, L: float = 1.0) -> float:
    """max over k != 0 of |k . u-hat(k)| / |k|, divided by max_k |u-hat(k)| (Sec. 4.1).

    The normalisation is global: a per-mode ratio is meaningless on modes whose
    amplitude is itself at the rounding level.
    """
    d = uhat.shape[0]
    ks = wavevectors(N, d, L)
    k2 = sum(k * k for k in ks)
    ku = np.abs(sum(ks[a] * uhat[a] for a in range(d)))
    un = np.sqrt(np.sum(np.abs(uhat) ** 2, axis=0))
    top = float(np.max(un))
    nz = k2 > 0
    if top == 0.0 or not np.any(nz):
        return 0.0
    return float(np.max(ku[nz] / np.sqrt(k2[nz]))) / top


def spread_at_modes(X: np.ndarray, c: np.ndarray, modes: np.ndarray, L: float = 1.0) -> np.ndarray:
    """The type-1 sum of Eq. force_spreading_quad at a list of integer modes (nk, d), one by one.

    Returns (ncomp, nk) complex. Used to check large transforms on sampled modes.
    """
    d, M = X.shape
    out = np.zeros((c.shape[0], modes.shape[0]), dtype=np.complex128)
    for q in range(modes.shape[0]):
        ph = np.zeros(M)
        for a in range(d):
            ph += TWO_PI / L * float(modes[q, a]) * X[a]
        e = np.exp(-1j * ph)
        out[:, q] = (c @ e) / L ** d
    return out
