"""Closed-form references of the two-dimensional validation problems (Sec. 5.2.2).

Channel of width D driven from rest by a uniform body force f0 along the channel,
no-slip walls, viscosity mu, density rho:

  Phi(t)  = sum_{k >= 0} 8 f0 / (mu lambda^3 (2k+1) pi) (1 - exp(-mu lambda^2 t / rho)),
            lambda = (2k+1) pi / D                                  (Eq. poiseuille_flux)
  Phi_eq  = f0 D^3 / (12 mu)                                        (Eq. steady_poiseuille_flux)
  D_e     = (12 mu Phi / f0)^(1/3), the channel width that carries flux Phi, and the
            effective boundary width Delta_e = D - D_e.

The oracle's channel pins (test_oracle_channel.py) check the oracle against these
formulas; they are written from the paper's equations and share nothing with the
oracle or the library.
"""
from __future__ import annotations

import math

import numpy as np


def poiseuille_flux(t, f0: float, mu: float, rho: float, D: float, nterms: int = 4000) -> np.ndarray:
    """Analytical flux of the started channel flow at times t (Eq. poiseuille_flux)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = 2.0 * np.arange(nterms, dtype=np.float64) + 1.0
    lam = n * math.pi / D
    amp = 8.0 * f0 / (mu * lam ** 3 * n * math.pi)
    return np.sum(amp[None, :] * -np.expm1(-(mu / rho) * lam[None, :] ** 2 * t[:, None]), axis=1)


def poiseuille_steady_flux(f0: float, mu: float, D: float) -> float:
    """Steady flux f0 D^3 / (12 mu) (Eq. steady_poiseuille_flux)."""
    return f0 * D ** 3 / (12.0 * mu)


def effective_width(flux: float, f0: float, mu: float) -> float:
    """Width D_e of the ideal channel that carries `flux` at equilibrium."""
    return (12.0 * mu * flux / f0) ** (1.0 / 3.0)


def embed_half_spectrum(H: np.ndarray, N2: int) -> np.ndarray:
    """Zero-pad a half spectrum (d, (N,) N, N//2) to N2 >= N modes per axis, keeping each
    integer mode m at its place (FFT order on the full axes, m_x = 0..N/2-1 on the last)."""
    d, N = H.shape[0], H.shape[1]
    out = np.zeros((d,) + (N2,) * (H.ndim - 2) + (N2 // 2,), dtype=H.dtype)
    i = np.arange(N)
    m = np.where(i < N // 2, i, i - N) % N2
    idx = np.ix_(*([np.arange(d)] + [m] * (H.ndim - 2) + [np.arange(N // 2)]))
    out[idx] = H
    return out


def half_spectrum_norm(H: np.ndarray) -> float:
    """L2 norm of the real field a half spectrum represents, up to the factor L^(d/2)
    (Parseval): entries with m_x > 0 stand for m and -m."""
    w = np.full(H.shape[-1], 2.0)
    w[0] = 1.0
    return float(np.sqrt(np.sum(w * np.abs(H) ** 2)))


def successive_errors(spectra) -> list:
    """Relative L2 difference of each solution from the next finer one (spectra listed
    from coarse to fine, each padded to the finer mode set)."""
    out = []
    for a, b in zip(spectra[:-1], spectra[1:]):
        N2 = b.shape[1]
        out.append(half_spectrum_norm(embed_half_spectrum(a, N2) - b) / half_spectrum_norm(b))
    return out
