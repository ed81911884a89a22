"""Pins of the oracle's lattice tables: the D3Q19 set (Sec. 5), the ball of the
smeared density (Sec. 3) and the contact shell with its quadrature weight
(the integral over k-hat of Eq. campoc).  Everything is checked against
properties fixed by mathematics, not against the oracle's own formulas."""
import itertools
import math

import numpy as np
import pytest

BALL_COUNTS = {3.0: 19, 4.0: 33, 6.0: 123, 8.0: 257}
SHELL_COUNTS = {3.0: 98, 4.0: 210, 6.0: 450, 8.0: 762}


def test_d3q19_moments(oracle_mod):
    c, w = oracle_mod.velocities()
    c = c.astype(float)
    assert len({tuple(v) for v in c.astype(int)}) == 19
    assert sorted(np.sum(c * c, axis=1).astype(int).tolist()) == [0] + [1] * 6 + [2] * 12
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    # third moments vanish, fourth moments isotropic: cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso, atol=1e-16)


def _brute(sigma, inside):
    R = int(math.ceil(sigma + 1))
    out = set()
    for v in itertools.product(range(-R, R + 1), repeat=3):
        if inside(v[0] ** 2 + v[1] ** 2 + v[2] ** 2):
            out.add(v)
    return out


@pytest.mark.parametrize("sigma", [3.0, 4.0, 6.0, 8.0])
def test_ball_and_shell_sets(oracle_mod, sigma):
    ball = {tuple(v) for v in oracle_mod.ball(sigma)}
    assert ball == _brute(sigma, lambda r2: r2 <= (sigma / 2) ** 2)
    assert len(ball) == BALL_COUNTS[sigma]
    e, _ = oracle_mod.shell(sigma)
    shell = {tuple(v) for v in e}
    assert shell == _brute(sigma, lambda r2: (sigma - 0.5) ** 2 < r2 <= (sigma + 0.5) ** 2)
    assert len(shell) == SHELL_COUNTS[sigma]


@pytest.mark.parametrize("sigma", [3.0, 4.0, 6.0, 8.0])
def test_shell_quadrature(oracle_mod, sigma):
    e, w = oracle_mod.shell(sigma)
    e = e.astype(float)
    L = np.linalg.norm(e, axis=1)
    k = e / L[:, None]
    # odd moments vanish (point symmetry); the second moment is isotropic and
    # normalised so that the discrete virial coefficient equals b = 2 pi sigma^3/3
    np.testing.assert_allclose(w * k.sum(axis=0), 0.0, atol=1e-13)
    M = sigma ** 2 * w * np.einsum("ma,mb->ab", k, e)
    np.testing.assert_allclose(M, np.eye(3) * 4.0 * math.pi * sigma ** 3 / 3.0, rtol=1e-13, atol=1e-10)
    # the weights integrate the unit sphere: sum w -> 4 pi
    assert abs(w * len(e) - 4 * math.pi) / (4 * math.pi) < 0.05


def test_shell_quadrature_converges(oracle_mod):
    errs = []
    for sigma in (4.0, 8.0):
        e, w = oracle_mod.shell(sigma)
        errs.append(abs(w * len(e) - 4 * math.pi))
    assert errs[1] < errs[0]
