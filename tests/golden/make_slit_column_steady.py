"""Writes slit_column_steady.txt: the FP64 oracle's steady slit Poiseuille
state of the 256 x 256 x 161 slit configuration (walls at z = 0 and 160,
sigma = 4, tau = 0.8, g_x = 1e-6, reduced densities 0.3 and 0.6 from a
uniform start).  A uniform start stays uniform in x and y, so the oracle runs
the 1 x 1 x 161 column (every shell and ball vector wraps onto it), which is
the same discrete state as any nx x ny cross-section.

Steady state: the relative change per step of the pore flux sum(n u_x),
checked every 100 steps, below 1e-12.  Reduced density 0.8 is beyond the
linear stability limit of the scheme's uniform fluid (about 0.65-0.7) and is
not part of the file.

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_slit_column_steady.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

NZ, SIGMA, TAU, GX = 161, 4.0, 0.8, 1e-6
DENSITIES = (0.3, 0.6)
TOL, CHECK, MAX_STEPS = 1e-12, 100, 2_000_000


def solve(n_star):
    n0 = n_star / SIGMA ** 3
    n = np.full((NZ, 1, 1), n0)
    n[0] = n[-1] = 0.0
    o = oracle.Oracle(1, 1, NZ, True, SIGMA, TAU, (GX, 0.0, 0.0))
    o.init(n)
    q_prev = None
    steps, res = 0, float("inf")
    while steps < MAX_STEPS:
        o.step(CHECK)
        steps += CHECK
        if o.unstable:
            raise RuntimeError("oracle unstable at n* = %g" % n_star)
        nn, uu = o.moments()
        q = float(np.sum(nn[1:-1] * uu[0, 1:-1]))
        if q_prev is not None:
            res = abs(q - q_prev) / (CHECK * abs(q))
            if res < TOL:
                break
        q_prev = q
    nn, uu = o.moments()
    return steps, res, nn[:, 0, 0], uu[0, :, 0, 0]


def main():
    oracle.build()
    out = os.path.join(HERE, "slit_column_steady.txt")
    lines = ["# FP64 oracle steady state of the slit configuration 256 x 256 x 161 (sigma = 4,",
             "# tau = 0.8, g_x = 1e-6, walls z = 0 and z = 160), from a uniform start, computed",
             "# on the 1 x 1 x 161 column by tests/golden/make_slit_column_steady.py (oracle only).",
             "# Steady state: relative pore-flux change per step < %g, checked every %d steps." % (TOL, CHECK)]
    for n_star in DENSITIES:
        steps, res, n, ux = solve(n_star)
        lines.append("# n_star %g steps %d residual %.3e" % (n_star, steps, res))
        lines.append("n_star: %r" % n_star)
        lines.append("steps: %d" % steps)
        lines.append("n: " + " ".join("%.17g" % v for v in n))
        lines.append("ux: " + " ".join("%.17g" % v for v in ux))
        print("n* %g: %d steps, residual %.2e" % (n_star, steps, res), flush=True)
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
