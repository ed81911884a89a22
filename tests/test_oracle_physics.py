"""Pins of the oracle against closed forms the paper and textbooks fix.

* Equation of state (Sec. 3 and Sec. 4: Enskog-like collisional pressure):
  for a long density wave the mean-field force is -grad P^c with
  P^c = kT b n^2 g2(n), b = 2 pi sigma^3 / 3; the ratio converges as q^2.
* Shear viscosity (Sec. 4, Eq. treotto with the cross-over term of
  Eq. extrapressure): decay of a transverse wave against the same analysis done
  with the lattice shell sums; interactions off gives nu q^2 with
  nu = kT (tau - 1/2) (BGK).
* Plane Poiseuille flow between smooth walls (Sec. 5) with interactions off:
  exact parabola at the bounce-back "magic" relaxation time
  (tau - 1/2)^2 = 3/16; exact curvature -g/nu at any tau.
* Contact theorem at a hard wall, p = kT n(contact), reached as sigma grows.
"""
import itertools
import math

import numpy as np
import pytest

KT = 1.0 / 3.0


def g_cs(chi):
    return (1 - chi / 2) / (1 - chi) ** 3


def dg_cs(chi):
    return (2.5 - chi) / (1 - chi) ** 4


def shell(sigma):
    R = int(math.floor(sigma + 0.5))
    e = np.array([v for v in itertools.product(range(-R, R + 1), repeat=3)
                  if (sigma - 0.5) ** 2 < v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= (sigma + 0.5) ** 2], float)
    L = np.linalg.norm(e, axis=1)
    return e, e / L[:, None], (4 * math.pi / 3) * sigma / np.sum(e[:, 2] ** 2 / L)


def eos_ratio(oracle_mod, L, sigma, n0, eps=1e-6):
    z = np.arange(L)
    q = 2 * math.pi / L
    n = (n0 * (1 + eps * np.sin(q * z))).reshape(L, 1, 1)
    o = oracle_mod.Oracle(1, 1, L, False, sigma, 1.0)
    o.init(n)
    _, C, _ = o.fields()
    amp = 2.0 / L * np.sum(C[2, :, 0, 0] * np.cos(q * z))
    b = 2 * math.pi * sigma ** 3 / 3
    chi = math.pi * sigma ** 3 * n0 / 6
    dPdn = KT * b * (2 * n0 * g_cs(chi) + n0 ** 2 * dg_cs(chi) * math.pi * sigma ** 3 / 6)
    return amp / (-dPdn * n0 * eps * q)


@pytest.mark.parametrize("sigma,nstar", [(4.0, 0.573), (3.0, 0.4)])
def test_equation_of_state_long_wave(oracle_mod, sigma, nstar):
    n0 = nstar / sigma ** 3
    r1 = eos_ratio(oracle_mod, 128, sigma, n0)
    r2 = eos_ratio(oracle_mod, 256, sigma, n0)
    assert abs(1 - r2) < abs(1 - r1) / 3.5          # q^2 convergence
    assert abs((4 * r2 - r1) / 3 - 1) < 2e-5        # Richardson limit is the EOS


def decay_rate(oracle_mod, L, sigma, nstar, tau, K, inter, steps=400, skip=100):
    z = np.arange(L)
    q = 2 * math.pi / L
    n = np.full((L, 1, 1), nstar / sigma ** 3)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = 1e-6 * np.sin(q * z)
    o = oracle_mod.Oracle(1, 1, L, False, sigma, tau, k_cross=K, interactions=inter)
    o.init(n, u)
    o.step(skip)
    t, a = [], []
    for s in range(steps - skip):
        o.step(1)
        _, uu = o.moments()
        t.append(s)
        a.append(2.0 / L * np.sum(uu[0, :, 0, 0] * np.sin(q * z)))
    return -np.polyfit(t, np.log(a), 1)[0]


def shear_theory(L, sigma, nstar, tau, K):
    """Linear decay rate of u_x = U sin(q z) with the discrete shell sums:
    kinetic nu q^2, cross-over (tau-1/2) K (kT/5) n g sigma^2 q S1 (A-term),
    collisional beta g n S2 (F^viscous)."""
    q = 2 * math.pi / L
    n0 = nstar / sigma ** 3
    e, k, w = shell(sigma)
    g = g_cs(math.pi * sigma ** 3 * n0 / 6)
    beta = 2 * sigma ** 2 * math.sqrt(KT / math.pi)
    S1 = np.sum(w * k[:, 2] * np.sin(q * e[:, 2]))
    S2 = np.sum(w * k[:, 0] ** 2 * (1 - np.cos(q * e[:, 2])))
    return KT * (tau - 0.5) * q * q, (tau - 0.5) * K * (KT / 5) * n0 * g * sigma ** 2 * q * S1, beta * g * n0 * S2


def test_shear_wave_bgk(oracle_mod):
    for L in (64, 128):
        r = decay_rate(oracle_mod, L, 4.0, 0.573, 1.0, 2.0, False)
        assert r == pytest.approx(KT * 0.5 * (2 * math.pi / L) ** 2, rel=1e-5)


def test_shear_wave_viscosity_with_cross_over(oracle_mod):
    L, sigma, nstar, tau = 128, 4.0, 0.573, 1.0
    kin, cross, coll = shear_theory(L, sigma, nstar, tau, 2.0)
    r2 = decay_rate(oracle_mod, L, sigma, nstar, tau, 2.0, True)
    r0 = decay_rate(oracle_mod, L, sigma, nstar, tau, 0.0, True)
    assert r2 == pytest.approx(kin + cross + coll, rel=1e-2)
    assert r0 == pytest.approx(kin + coll, rel=1e-2)
    assert (r2 - r0) == pytest.approx(cross, rel=3e-2)
    # continuum limit of the same terms (Sec. 4): cross-over = kinetic * (8 pi/15) n* g (K=2)
    g = g_cs(math.pi * nstar / 6)
    assert cross / kin == pytest.approx((8 * math.pi / 15) * nstar * g, rel=0.03)


@pytest.mark.parametrize("tau", [0.5 + math.sqrt(3) / 4, 1.0])
def test_poiseuille_bgk(oracle_mod, tau):
    nz, g = 21, 1e-6
    o = oracle_mod.Oracle(1, 1, nz, True, 4.0, tau, (g, 0, 0), interactions=False)
    o.init(np.full((nz, 1, 1), 0.01))
    o.step(20000)
    _, uu = o.moments()
    ux = uu[0, 1:-1, 0, 0]
    nu = KT * (tau - 0.5)
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    np.testing.assert_allclose(d2, -g / nu, rtol=1e-9)
    if abs((tau - 0.5) ** 2 - 3 / 16) < 1e-12:
        z = np.arange(1, nz - 1)
        np.testing.assert_allclose(ux, g / (2 * nu) * (z - 0.5) * (nz - 1.5 - z), rtol=1e-9)


def contact_ratio(oracle_mod, sigma, nstar):
    nz = int(24 * sigma) + 1
    n0 = nstar / sigma ** 3
    o = oracle_mod.Oracle(1, 1, nz, True, sigma, 1.0)
    o.init(np.full((nz, 1, 1), n0))
    prev = None
    for _ in range(60):
        o.step(250)
        prof = o.moments()[0][:, 0, 0]
        if prev is not None and np.abs(prof - prev).max() / n0 < 1e-8:
            break
        prev = prof
    mid = prof[nz // 2]
    chi = math.pi * sigma ** 3 * mid / 6
    p = KT * mid * (1 + 2 * math.pi * sigma ** 3 / 3 * mid * g_cs(chi))
    return KT * prof[1] / p


def test_contact_theorem(oracle_mod):
    r4 = contact_ratio(oracle_mod, 4.0, 0.3)
    r6 = contact_ratio(oracle_mod, 6.0, 0.3)
    assert r4 < r6 < 1.0                       # deficit shrinks with sigma
    assert abs((6 * r6 - 4 * r4) / 2 - 1) < 0.03   # O(1/sigma) extrapolation


def test_nbar_relaxation_mode_viscosity(oracle_mod):
    """omega0 proportional to n g2 (Sec. 4): with the relaxation time scaled by
    n_ref g2(n_ref) / (nbar g2(nbar)), a uniform fluid of density n relaxes
    exactly like the constant mode at tau_eff; with n_ref = n, tau_eff = tau."""
    L, sigma, nstar, tau = 64, 4.0, 0.4, 1.0
    n0 = nstar / sigma ** 3
    q = 2 * math.pi / L
    z = np.arange(L)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = 1e-6 * np.sin(q * z)

    def rate(**kw):
        o = oracle_mod.Oracle(1, 1, L, False, sigma, kw.pop("tau"), interactions=False, **kw)
        o.init(np.full((L, 1, 1), n0), u)
        o.step(50)
        a0 = 2.0 / L * np.sum(o.moments()[1][0, :, 0, 0] * np.sin(q * z))
        o.step(200)
        a1 = 2.0 / L * np.sum(o.moments()[1][0, :, 0, 0] * np.sin(q * z))
        return math.log(a0 / a1) / 200

    chi = lambda n: math.pi * sigma ** 3 * n / 6
    tau_eff = 0.5 + (tau - 0.5) * (2 * n0 * g_cs(chi(2 * n0))) / (n0 * g_cs(chi(n0)))
    assert rate(tau=tau, omega_mode="nbar", n_ref=n0) == pytest.approx(rate(tau=tau), rel=1e-9)
    # without n_ref the reference is the initial fluid mean, here n0
    assert rate(tau=tau, omega_mode="nbar") == pytest.approx(rate(tau=tau), rel=1e-9)
    assert rate(tau=tau, omega_mode="nbar", n_ref=2 * n0) == pytest.approx(rate(tau=tau_eff), rel=1e-9)
    assert rate(tau=tau_eff) == pytest.approx(KT * (tau_eff - 0.5) * q * q, rel=0.03)


def test_nbar_mode_default_reference_is_the_fluid_mean(oracle_mod):
    """In a slit the default reference density of the nbar relaxation mode is
    the initial mean over the fluid planes (the solid planes, whatever the
    input holds there, do not count): the same run as with that mean given."""
    nx, ny, nz = 6, 5, 17
    rng = np.random.default_rng(4)
    n = (0.4 / 64) * (1 + 0.02 * rng.standard_normal((nz, ny, nx)))
    n[0], n[-1] = 0.03, 0.05                   # ignored: solid planes
    mean = n[1:-1].mean()
    runs = []
    for kw in ({}, {"n_ref": mean}, {"n_ref": n.mean()}):
        o = oracle_mod.Oracle(nx, ny, nz, True, 4.0, 0.9, (1e-5, 0.0, 0.0), omega_mode="nbar", **kw)
        o.init(n)
        o.step(5)
        runs.append(o.moments()[1])
    scale = np.abs(runs[0]).max()
    assert np.abs(runs[0] - runs[1]).max() < 1e-12 * scale     # the two means differ in summation order
    assert np.abs(runs[0] - runs[2]).max() > 1e-2 * scale      # the all-node mean: a different run
