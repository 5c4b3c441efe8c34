"""Writes the regression fixtures of this folder.  It calls only the FP64
oracle (oracle/) and the seeded input generators, never the CUDA path.

    python tests/golden/make_golden.py

oracle_2d32_rk4.txt: energy and enstrophy of the 2D random field of seed 0
(32^2, k0 = 3, E = 0.5) after 0, 10 and 20 Lawson IF-RK4 steps (nu = 0.005,
dt = 0.02, no forcing), and the real and imaginary parts of three fixed
modes after 20 steps.  These guard the oracle against unintended changes;
they are not pins (the pins are closed forms, brute force and invariants,
tests/test_oracle_*.py).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1807_01769_gb300 import inputs  # noqa: E402

MODES = [(1, 2), (5, 3), (20, 7)]  # (row, kx) of the truncated (c, h) layout


def compute():
    n, nu, dt = 32, 0.005, 0.02
    u = inputs.random_vorticity_2d(n, seed=0, k0=3.0)
    lines = []
    for k in (0, 10, 20):
        s = oracle.step(2, n, nu, dt, k, u) if k else u
        e, om = oracle.diagnostics(2, n, s)
        lines.append(f"steps={k} energy={float(e)!r} enstrophy={float(om)!r}")
    for r, kx in MODES:
        v = s[r, kx]
        lines.append(f"mode={r},{kx} re={float(v.real)!r} im={float(v.imag)!r}")
    return lines


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_2d32_rk4.txt"), "w") as f:
        f.write("\n".join(compute()) + "\n")
