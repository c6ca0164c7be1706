"""Closed-form references of the two-dimensional validation problems (Sec. 5.2.2).

Channel of width D driven from rest by a uniform body force f0 along the channel,
no-slip walls, viscosity mu, density rho:

  Phi(t)  = sum_{k >= 0} 8 f0 / (mu lambda^3 (2k+1) pi) (1 - exp(-mu lambda^2 t / rho)),
            lambda = (2k+1) pi / D                                  (Eq. poiseuille_flux)
  Phi_eq  = f0 D^3 / (12 mu)                                        (Eq. steady_poiseuille_flux)
  D_e     = (12 mu Phi / f0)^(1/3), the channel width that carries flux Phi, and the
            effective boundary width Delta_e = D - D_e.

These are host-side formulas for reporting; the flux of a computed velocity comes
from the library (fsib_band_flux).
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
