"""Pins of the contact value g2 (Sec. 3) and of the one-node collision
(Sec. 5 step 3: Eq. relaxationtime, Eq. SMDB, Eq. eq:dufty2)."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("chi", [1e-4, 0.05, 0.157, 0.262, 0.3, 0.419])
def test_carnahan_starling_contact_value(oracle_mod, chi):
    # g2 from the Carnahan-Starling compressibility factor Z = 1 + 4 chi g2
    Z = (1 + chi + chi ** 2 - chi ** 3) / (1 - chi) ** 3
    assert oracle_mod.closure("CS", chi) == pytest.approx((Z - 1) / (4 * chi), rel=1e-12)


@pytest.mark.parametrize("kind", ["CS", "PY"])
def test_second_virial_coefficient_of_g2(oracle_mod, kind):
    # exact low-density expansion of the hard-sphere contact value: 1 + 5/2 chi + O(chi^2)
    for chi in (1e-3, 1e-4):
        g = oracle_mod.closure(kind, chi)
        assert abs((g - 1.0) / chi - 2.5) < 10 * chi
    assert oracle_mod.closure("ONE", 0.3) == 1.0


def test_collision_moments(oracle_mod):
    """Guo second-order forcing identities: the collision conserves mass, adds
    F to the momentum, and its second moment relaxes toward the equilibrium
    stress with the force and A-term sources (factor 1 - omega/2)."""
    c, w = oracle_mod.velocities()
    c = c.astype(float)
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 0.01 * (1 + 0.2 * rng.random())
        u0 = 0.05 * rng.standard_normal(3)
        feq = w * n * (1 + 3 * c @ u0 + 4.5 * (c @ u0) ** 2 - 1.5 * u0 @ u0)
        fin = feq * (1 + 0.01 * rng.standard_normal(19))
        F = 1e-4 * rng.standard_normal(3)
        A6 = 1e-4 * rng.standard_normal(6)
        omega = 1.0 / (0.6 + rng.random())
        K = 2.0
        fout = oracle_mod.collide_node(fin, F, A6, omega, K)
        n_in = fin.sum()
        j_in = fin @ c
        assert fout.sum() == pytest.approx(n_in, rel=1e-14)
        np.testing.assert_allclose(fout @ c, j_in + F, rtol=0, atol=1e-16)
        u = (j_in + 0.5 * F) / n_in
        Pi_in = np.einsum("q,qa,qb->ab", fin, c, c)
        Pi_eq = n_in * np.eye(3) / 3.0 + n_in * np.outer(u, u)
        A = np.array([[A6[0], A6[3], A6[4]], [A6[3], A6[1], A6[5]], [A6[4], A6[5], A6[2]]])
        At = A - np.trace(A) / 3 * np.eye(3)
        src = np.outer(u, F) + np.outer(F, u) + K * At
        expect = (1 - omega) * Pi_in + omega * Pi_eq + (1 - omega / 2) * src
        np.testing.assert_allclose(np.einsum("q,qa,qb->ab", fout, c, c), expect, rtol=1e-12, atol=1e-17)


def test_collision_rest_state_is_fixed_point(oracle_mod):
    c, w = oracle_mod.velocities()
    fin = 0.0078 * w
    fout = oracle_mod.collide_node(fin, np.zeros(3), np.zeros(6), 1.0, 2.0)
    np.testing.assert_allclose(fout, fin, rtol=1e-15)
