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


def test_column_equals_uniform_slab(oracle_mod):
    """A state uniform in x and y is the same on a 1 x 1 x nz column (every
    shell and ball vector wraps onto it) as on a wider slab; the steady slit
    fixtures rely on it."""
    nz, sigma = 21, 4.0
    z = np.arange(nz)
    prof = (0.45 / 64) * (1.0 + 0.05 * np.sin(2 * np.pi * z / (nz - 2)))
    prof[0] = prof[-1] = 0.0
    ux = 1e-4 * np.sin(np.pi * z / (nz - 1))
    ux[0] = ux[-1] = 0.0
    out = []
    for nxy in (1, 5):
        n = np.broadcast_to(prof[:, None, None], (nz, nxy, nxy)).copy()
        u = np.zeros((3, nz, nxy, nxy))
        u[0] = ux[:, None, None]
        o = oracle_mod.Oracle(nxy, nxy, nz, True, sigma, 0.9, (1e-6, 0, 0))
        o.init(n, u)
        o.step(30)
        nn, uu = o.moments()
        out.append((nn[:, 0, 0], uu[:, :, 0, 0]))
        assert np.abs(nn - nn[:, :1, :1]).max() == 0.0 and np.abs(uu - uu[:, :, :1, :1]).max() == 0.0
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-14)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=0, atol=1e-14 * np.abs(out[1][1]).max())
