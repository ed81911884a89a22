"""Pins of the oracle against the shear-viscosity numbers printed in Sec. 4
(tests/golden/sec4_shear_viscosity.txt).

With the collision frequency of Sec. 4, omega0 = 3.2 n sigma^2 g2 sqrt(pi kT/m),
taken as the lattice relaxation rate (tau - 1/2 = 1/omega0), the cross-over
part of the measured viscosity must equal Enskog's 0.8 b n eta0 (the paper's
own check of the factor of the A-term), and the collisional part the paper's
(4/15) sqrt(m pi kT) n^2 sigma^4 g2.  The oracle's shell quadrature is
anisotropic by a few per cent at sigma = 4, which sets the tolerances
(measured: cross-over 0.808 against 0.8; K = 1 would give 0.40)."""
import math
import os

import pytest

from test_oracle_physics import KT, decay_rate, g_cs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sec4_shear_viscosity.txt")


def golden():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split(":")
                vals[k.strip()] = float(v)
    return vals


def test_cross_over_and_collisional_viscosity_match_sec4():
    import oracle
    oracle.build()
    gv = golden()
    L, sigma, nstar = 128, 4.0, 0.573
    n0 = nstar / sigma ** 3
    g = g_cs(math.pi * nstar / 6)
    omega0 = gv["omega0_coefficient"] * n0 * sigma ** 2 * g * math.sqrt(math.pi * KT)
    tau = 0.5 + 1.0 / omega0
    q = 2 * math.pi / L
    r2 = decay_rate(oracle, L, sigma, nstar, tau, 2.0, True)      # with cross-over
    r0 = decay_rate(oracle, L, sigma, nstar, tau, 0.0, True)      # without
    kin = KT * (tau - 0.5) * q * q
    eta0 = gv["eta0_coefficient"] / sigma ** 2 * math.sqrt(KT / math.pi)
    b = 2 * math.pi * sigma ** 3 / 3
    # u decays at (eta / n) q^2: dynamic viscosities per part
    eta_cross = n0 * (r2 - r0) / (q * q)
    eta_coll = n0 * (r0 - kin) / (q * q)
    assert eta_cross / (eta0 * b * n0) == pytest.approx(gv["enskog_cross_over"], rel=0.02)
    paper_coll = gv["collisional_factor"] * math.sqrt(math.pi * KT) * n0 ** 2 * sigma ** 4 * g
    assert eta_coll == pytest.approx(paper_coll, rel=0.01)
    # the kinetic part with this omega0 is eta0 / g2 (the paper's form of Enskog's 1.016 / g2)
    assert n0 * KT * (tau - 0.5) * g / eta0 == pytest.approx(1.0, rel=1e-12)
    # cross-over factor of Eq. treotto: (8 pi / 15) n sigma^3 g2 times the kinetic part
    assert eta_cross / (n0 * KT / omega0) == pytest.approx(
        gv["cross_over_factor_over_pi"] * math.pi * nstar * g, rel=0.03)
