"""Exact invariants of the discrete scheme, checked on the oracle:
mass conservation (Eq. continuity), momentum balance with the pair
antisymmetry of C (Eq. gradient: C is the divergence of a stress, so its
lattice sum vanishes), and a uniform state at rest staying at rest."""
import numpy as np
import pytest

from paper_1304_7880_gb300 import synth


def _total_momentum(o):
    f = o.populations()
    import oracle
    c, _ = oracle.velocities()
    return np.einsum("qzyx,qa->a", f, c.astype(float))


def test_mass_conserved_in_slit(oracle_mod):
    p, n, u = synth.slit_poiseuille(4, 4, 21, 0.5, 4.0, 1.0, 1e-5, seed=11)
    o = oracle_mod.Oracle(**p)
    o.init(n, u)
    m0 = o.moments()[0].sum()
    o.step(60)
    m1 = o.moments()[0].sum()
    assert abs(m1 - m0) / m0 < 1e-13
    assert not o.unstable


@pytest.mark.parametrize("closure", ["CS", "ONE"])
def test_momentum_balance_periodic(oracle_mod, closure):
    """sum_r j(t+1) = sum_r j(t) + g sum_r n: collisional forces cancel pairwise."""
    sigma = 3.0
    n0 = synth.reduced_to_density(0.5, sigma)
    n, u = synth.uniform_with_noise(7, 6, 9, n0, 2e-2, 5, False)
    rng = np.random.default_rng(3)
    u = 1e-3 * rng.standard_normal(u.shape)
    g = (2e-6, -1e-6, 3e-6)
    o = oracle_mod.Oracle(7, 6, 9, False, sigma, 0.9, g, closure=closure)
    o.init(n, u)
    P0 = _total_momentum(o)
    mass = o.moments()[0].sum()
    nsteps = 25
    o.step(nsteps)
    P1 = _total_momentum(o)
    scale = np.abs(o.populations()).sum() * 1e-14
    np.testing.assert_allclose(P1 - P0, nsteps * mass * np.array(g), rtol=0, atol=scale)


def test_fields_sum_to_zero(oracle_mod):
    """Lattice sum of C vanishes (pair antisymmetry with the midpoint g2)."""
    sigma = 4.0
    n0 = synth.reduced_to_density(0.5, sigma)
    n, u = synth.uniform_with_noise(9, 9, 9, n0, 5e-2, 8, False)
    rng = np.random.default_rng(4)
    u = 1e-3 * rng.standard_normal(u.shape)
    o = oracle_mod.Oracle(9, 9, 9, False, sigma, 1.0)
    o.init(n, u)
    _, C, _ = o.fields()
    scale = np.abs(C).sum() * 1e-13
    np.testing.assert_allclose(C.sum(axis=(1, 2, 3)), 0.0, atol=scale)


def test_uniform_rest_state_is_stationary(oracle_mod):
    """A uniform periodic state at rest is exactly stationary (sum_e w khat = 0
    and nbar = n for uniform n)."""
    sigma = 4.0
    n0 = synth.reduced_to_density(0.5, sigma)
    n = np.full((10, 10, 10), n0)
    o = oracle_mod.Oracle(10, 10, 10, False, sigma, 1.0)
    o.init(n)
    f0 = o.populations()
    o.step(20)
    np.testing.assert_allclose(o.populations(), f0, rtol=1e-13)
