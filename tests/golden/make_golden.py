"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Inputs come from the seeded generators; outputs come only from oracle/.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import spectral as sp  # noqa: E402
from oracle import stepper as st  # noqa: E402
from paper_2302_08694_gb300 import workloads as wl  # noqa: E402


def c2l(a):
    a = np.asarray(a)
    return {"re": a.real.ravel().tolist(), "im": a.imag.ravel().tolist(), "shape": list(a.shape)}


def main():
    out = {"note": "oracle outputs on tiny seeded inputs; regression guard for the oracle"}
    # 2D quasi-static Stokes: ellipse (0.3, 0.2), K = 1, mu = 1, N = 8, M = 16, two steps
    rng = np.random.default_rng(101)
    X = wl.ellipse(16, 0.3, 0.2, rng.uniform(0, 1, 2))
    force = st.curve_model(1.0)
    Xs = X.copy()
    for _ in range(2):
        Xs = st.stokes_step(Xs, force, 8, 1.0, 1e-3)
    out["stokes2d"] = {"X0": X.tolist(), "N": 8, "mu": 1.0, "dt": 1e-3, "nsteps": 2,
                       "K": 1.0, "X": Xs.tolist()}
    # 3D type-1 sum: N = 4, M = 5
    rng = np.random.default_rng(102)
    Y = rng.uniform(0, 1, (3, 5))
    c = rng.standard_normal((3, 5))
    f = sp.spread_direct(Y, c, 4)
    out["spread3d"] = {"X": Y.tolist(), "c": c.tolist(), "N": 4,
                       "fhat_half": c2l(sp.full_to_half(f, 4))}
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
