"""The oracle against the stored fixtures under tests/golden/ (cited paper values and a
regression record of tiny oracle runs)."""
import json
import math
import os

import numpy as np

from oracle import spectral as sp
from oracle import stepper as st

G = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_values_normal_circle_and_sinusoid():
    pv = json.load(open(os.path.join(G, "paper_values.json")))
    nc = pv["normal_force_circle"]
    Nb, r, mu = nc["Nb"], nc["r_over_L"] * nc["L"], nc["mu"]
    th = 2 * np.pi * np.arange(Nb) / Nb
    X = 0.5 + r * np.stack([np.cos(th), np.sin(th)])
    c = nc["F"] * (2 * np.pi / Nb) * np.stack([np.cos(th), np.sin(th)])
    for N in nc["N_below_transition"]:
        U = st.stokes_velocity(X, lambda Y: c, N, mu)
        assert np.max(np.abs(U)) <= 100 * nc["machine_error"]
    amp = pv["stokes_sinusoid"]["amplitude_times_mu_over_L2"]
    assert abs(amp - 1 / (4 * math.pi ** 2)) < 1e-17


def test_oracle_tiny_regression():
    g = json.load(open(os.path.join(G, "oracle_tiny.json")))
    s = g["stokes2d"]
    X = np.array(s["X0"])
    force = st.curve_model(s["K"])
    for _ in range(s["nsteps"]):
        X = st.stokes_step(X, force, s["N"], s["mu"], s["dt"])
    assert np.max(np.abs(X - np.array(s["X"]))) <= 1e-14
    p = g["spread3d"]
    f = sp.full_to_half(sp.spread_direct(np.array(p["X"]), np.array(p["c"]), p["N"]), p["N"])
    ref = (np.array(p["fhat_half"]["re"]) + 1j * np.array(p["fhat_half"]["im"])).reshape(p["fhat_half"]["shape"])
    assert np.max(np.abs(f - ref)) <= 1e-14
