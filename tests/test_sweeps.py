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


@pytest.mark.parametrize("sigma", [3.0, 4.0, 6.0, 8.0])
def test_compact_shell_viscosity_is_the_continuum_form(sigma):
    """With the compact shell, whose moment sum_e w_e khat_x^2 e_z^2 is the
    continuum 4 pi sigma^2 / 15, the closed form is Sec. 4's continuum value
    eta = n [kT (tau-1/2) + (tau-1/2) K kT n g2 4 pi sigma^3/15
             + beta g2 n 2 pi sigma^2/15]; the full shell's differs from it only
    by its fourth-moment anisotropy (a few per cent of the collisional part)."""
    from paper_1304_7880_gb300 import build, sweeps, synth
    build.build()
    kT, tau, chi = 1.0 / 3.0, 1.0, 0.3
    n = synth.packing_to_density(chi, sigma)
    g2 = sweeps.contact_value(chi)
    beta = 2 * sigma ** 2 * math.sqrt(kT / math.pi)
    cont = n * (kT * (tau - 0.5) + (tau - 0.5) * 2 * kT * n * g2 * 4 * math.pi * sigma ** 3 / 15
                + beta * g2 * n * 2 * math.pi * sigma ** 2 / 15)
    assert sweeps.bulk_shear_viscosity(n, sigma, tau, 2.0, "compact") == pytest.approx(cont, rel=1e-12)
    assert sweeps.bulk_shear_viscosity(n, sigma, tau, 2.0, "full") == pytest.approx(cont, rel=0.05)
