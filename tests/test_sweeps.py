"""The pore-viscosity sweep's bulk normalisation (host only): the closed-form
long-wave shear viscosity equals the finite-wavenumber theory of the shear-wave
decay (the one the oracle's measured decay rates are pinned to) as q -> 0."""
import math

import pytest

from test_oracle_physics import shear_theory


@pytest.mark.parametrize("sigma,chi,tau", [(4.0, 0.11, 1.0), (4.0, 0.32, 1.0), (3.0, 0.3, 0.8), (6.0, 0.2, 1.2)])
def test_bulk_viscosity_is_the_long_wave_limit(sigma, chi, tau):
    from paper_1304_7880_gb300 import build, sweeps, synth
    build.build()
    n = synth.packing_to_density(chi, sigma)
    L = 1 << 14
    q = 2 * math.pi / L
    kin, cross, coll = shear_theory(L, sigma, n * sigma ** 3, tau, 2.0)
    assert sweeps.bulk_shear_viscosity(n, sigma, tau) == pytest.approx(n * (kin + cross + coll) / q ** 2, rel=1e-6)
