"""Pins of the oracle's energy-equation fields (oracle.thermal_fields): Q of
Eq. campob1, B of Eq. campos and the thermal force F^T of Eq. thermalforce on
a prescribed temperature field T (k_B T in lattice units, m = 1).

The paper's numerics are isothermal (Sec. 5); these fields are its energy
equation's collisional terms, checked against what the paper and the
mathematics fix:

* a uniform T and a fluid at rest give Q = B = F^T = 0;
* long-wave limits on a uniform fluid, T = T0 + a sin(kappa x), extrapolated
  to kappa -> 0 (Richardson, errors O(kappa^4)):
  - F^T_x -> -(2 pi / 3) sigma^3 g2 n dT/dx, the continuum integral of
    Eq. thermalforce (the shell's moment sum_e w khat_x e_x equals
    4 pi sigma / 3 exactly by the virial normalisation);
  - B_x -> -2 T n (4 pi / 3) sigma^3 g2 n dT/dx (Eq. campos);
  - Q -> lambda_c d2T/dx2 with lambda_c the collisional term of
    Eq. thermalcond, (2/3) sqrt(pi T) g2 n^2 sigma^4, times the shell's
    second-moment ratio sum_e w e_x^2 / (4 pi sigma^2 / 3): 1.048, 1.020,
    1.022, 1.004 at sigma = 3, 4, 6, 8 (the shell's radial width, so the
    discrete collisional conductivity exceeds the paper's by that much);
* momentum balance: the mean-field force at the local temperature
  (-T sigma^2 sum_e w khat g2 n(r+e)) and F^T together carry (T + T')/2 per
  pair, so n (F^mf_T + F^T) sums to zero over a periodic box and over a slit,
  for any n and T.
"""
import numpy as np
import pytest


def cs_g2(chi):
    return (1.0 - 0.5 * chi) / (1.0 - chi) ** 3


def _column(oracle_mod, L, sigma, nstar, T):
    o = oracle_mod.Oracle(L, 1, 1, False, sigma, 1.0, (0.0, 0.0, 0.0))
    o.init(np.full((1, 1, L), nstar / sigma ** 3))
    return o.thermal_fields(T.reshape(1, 1, L))


def test_uniform_temperature_at_rest_gives_no_fields(oracle_mod):
    rng = np.random.default_rng(3)
    n = (0.4 / 27) * (1 + 0.05 * rng.standard_normal((6, 7, 9)))
    o = oracle_mod.Oracle(9, 7, 6, False, 3.0, 1.0, (0.0, 0.0, 0.0))
    o.init(n)
    Qf, B, FT = o.thermal_fields(np.full(n.shape, 0.4))
    assert np.abs(Qf).max() == 0 and np.abs(B).max() == 0 and np.abs(FT).max() == 0


def _long_wave(oracle_mod, sigma, nstar, which, T0=0.35, a=1e-4):
    """Coefficient of the field's long-wave limit, Richardson-extrapolated."""
    vals = []
    for L in (256, 512):
        kappa = 2 * np.pi / L
        x = np.arange(L)
        T = T0 + a * np.sin(kappa * x)
        Qf, B, FT = _column(oracle_mod, L, sigma, nstar, T)
        if which == "FT":      # at x = 0: T = T0, dT/dx = a kappa
            vals.append(FT[0, 0, 0, 0] / (a * kappa))
        elif which == "B":
            vals.append(B[0, 0, 0, 0] / (a * kappa))
        else:                  # at x = L/4: T = T0 + a, d2T/dx2 = -a kappa^2
            vals.append(Qf[0, 0, L // 4] / (-a * kappa ** 2) / np.sqrt(T0 + a))
    return (4 * vals[1] - vals[0]) / 3


@pytest.mark.parametrize("sigma", [3.0, 4.0])
def test_thermal_force_long_wave_limit(oracle_mod, sigma):
    nstar = 0.4
    n = nstar / sigma ** 3
    g2 = cs_g2(np.pi * sigma ** 3 / 6 * n)
    got = _long_wave(oracle_mod, sigma, nstar, "FT")
    want = -(2 * np.pi / 3) * sigma ** 3 * g2 * n
    assert abs(got / want - 1) < 1e-6


@pytest.mark.parametrize("sigma", [3.0, 4.0])
def test_heat_flux_correction_long_wave_limit(oracle_mod, sigma):
    nstar, T0 = 0.4, 0.35
    n = nstar / sigma ** 3
    g2 = cs_g2(np.pi * sigma ** 3 / 6 * n)
    got = _long_wave(oracle_mod, sigma, nstar, "B", T0=T0)
    want = -2 * T0 * n * (4 * np.pi / 3) * sigma ** 3 * g2 * n
    assert abs(got / want - 1) < 1e-6


@pytest.mark.parametrize("sigma", [3.0, 4.0])
def test_collisional_conduction_is_the_thermalcond_term(oracle_mod, sigma):
    """Q / sqrt(T) on a sinusoidal T -> the collisional conductivity of
    Eq. thermalcond divided by sqrt(T), with the shell's second moment."""
    nstar = 0.4
    n = nstar / sigma ** 3
    g2 = cs_g2(np.pi * sigma ** 3 / 6 * n)
    e, w = oracle_mod.shell(sigma)
    m2 = float(np.sum(w * e[:, 0] ** 2))                   # sum_e w e_x^2
    ratio = m2 / (4 * np.pi * sigma ** 2 / 3)
    lam_paper = (2.0 / 3.0) * np.sqrt(np.pi) * g2 * n ** 2 * sigma ** 4   # / sqrt(T)
    got = _long_wave(oracle_mod, sigma, nstar, "Q")
    assert abs(got / (lam_paper * ratio) - 1) < 1e-6
    assert 1.0 < ratio < 1.05


@pytest.mark.parametrize("walls", [False, True])
def test_mean_field_and_thermal_force_conserve_momentum(oracle_mod, walls):
    rng = np.random.default_rng(11)
    nx, ny, nz = 10, 9, 12
    n = (0.4 / 27) * (1 + 0.1 * rng.standard_normal((nz, ny, nx)))
    if walls:
        n[0] = n[-1] = 0.0
    T = 0.33 * (1 + 0.2 * rng.standard_normal((nz, ny, nx)))
    o = oracle_mod.Oracle(nx, ny, nz, walls, 3.0, 1.0, (0.0, 0.0, 0.0))
    o.init(n)                       # at rest: C = n F^mf at k_B T = 1/3
    _, C, _ = o.fields()
    _, _, FT = o.thermal_fields(T)
    terms = 3.0 * T * C + n * FT     # n (F^mf at the local T + F^T)
    total = terms.reshape(3, -1).sum(axis=1)
    scale = np.abs(terms).reshape(3, -1).sum(axis=1)
    assert np.all(np.abs(total) < 1e-13 * scale), (total, scale)
    # and the thermal force alone does not balance (the check has teeth)
    assert np.abs((n * FT).reshape(3, -1).sum(axis=1)).max() > 1e-6 * scale.max()
