"""Pins of the oracle's compact contact shell (a quadrature of this library for
the integral over k-hat of Eq. campoc; the paper gives none).

The rule: the union of two or three cubic orbits of the full shell
(sigma - 1/2)^2 < |e|^2 <= (sigma + 1/2)^2, one positive weight per orbit, with
  sigma^2 sum_e w_e khat_z e_z = 4 pi sigma^3 / 3      (virial coefficient b)
  sum_e w_e khat_x^2 e_z^2     = 4 pi sigma^2 / 15     (viscosity moment)
  sum_e w_e khat_z^2 e_z^2     = 3 sum_e w_e khat_x^2 e_z^2   (isotropy)
and, of all such unions, the fewest vectors (then the smallest
sum (|e|^2 - sigma^2)^2, then the first in orbit order).

Each pin checks the oracle against mathematics, not its own formulas:
the moment conditions and the full fourth-rank isotropy by direct sums, the
cubic symmetry of the set, the selection by an independent numpy brute force
over all unions, the shell sums by FFT convolution, the equation of state in
the long-wave limit, the shear viscosity against the continuum closed form of
Sec. 4 (which the compact moments reproduce exactly as q -> 0), and the exact
conservation of mass and momentum.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

KT = 1.0 / 3.0
SIGMAS = [2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 6.0, 7.0, 8.0]


def g_cs(chi):
    return (1 - chi / 2) / (1 - chi) ** 3


def dg_cs(chi):
    return (2.5 - chi) / (1 - chi) ** 4


def cubic_ops():
    ops = []
    for p in itertools.permutations(range(3)):
        for s in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3), dtype=int)
            for r in range(3):
                M[r, p[r]] = s[r]
            ops.append(M)
    return ops


def brute_force_rule(sigma):
    """Independent restatement of the selection: every union of 2 or 3 cubic
    orbits of the full shell, weights by least squares, kept if the three
    conditions hold and every weight is positive."""
    R = int(math.floor(sigma + 0.5))
    vecs = [v for v in itertools.product(range(-R, R + 1), repeat=3)
            if (sigma - 0.5) ** 2 < v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= (sigma + 0.5) ** 2]
    orbits = {}
    for v in vecs:
        orbits.setdefault(tuple(sorted(abs(c) for c in v)), []).append(v)
    keys = sorted(orbits, key=lambda k: (k[0] ** 2 + k[1] ** 2 + k[2] ** 2, k))
    cols = []
    for k in keys:
        e = np.array(orbits[k], float)
        L = np.linalg.norm(e, axis=1)
        kh = e / L[:, None]
        cols.append([np.sum(kh[:, 2] * e[:, 2]), np.sum(kh[:, 0] ** 2 * e[:, 2] ** 2),
                     np.sum(kh[:, 2] ** 2 * e[:, 2] ** 2 - 3 * kh[:, 0] ** 2 * e[:, 2] ** 2)])
    rhs = np.array([4 * math.pi * sigma / 3, 4 * math.pi * sigma ** 2 / 15, 0.0])
    best = None
    for k in (1, 2, 3):
        for sub in itertools.combinations(range(len(keys)), k):
            A = np.array([cols[j] for j in sub]).T
            w = np.linalg.lstsq(A, rhs, rcond=None)[0]
            mag = np.abs(A * w).sum(axis=1) + np.abs(rhs)
            if np.any(np.abs(A @ w - rhs) > 1e-9 * mag) or not np.all(w > 1e-3 * w.max()):
                continue
            assert k > 1, "a single orbit satisfying all three conditions"
            n = sum(len(orbits[keys[j]]) for j in sub)
            spread = sum(len(orbits[keys[j]]) * (sum(c * c for c in keys[j]) - sigma ** 2) ** 2 for j in sub)
            if best is None or n < best[0] or (n == best[0] and spread < best[1] - 1e-9 * (1 + best[1])):
                best = (n, spread, {v: w[i] for i, j in enumerate(sub) for v in orbits[keys[j]]})
    return None if best is None else best[2]


@pytest.mark.parametrize("sigma", SIGMAS)
def test_compact_moments_and_symmetry(oracle_mod, sigma):
    e, w = oracle_mod.shell_compact(sigma)
    ef = e.astype(float)
    L = np.linalg.norm(ef, axis=1)
    k = ef / L[:, None]
    assert np.all(w > 0)
    full = {tuple(v) for v in oracle_mod.shell(sigma)[0]}
    assert {tuple(v) for v in e} <= full and len({tuple(v) for v in e}) == len(e)
    # cubic symmetry: the set is closed under the 48 operations, one weight per orbit
    wt = {tuple(v): x for v, x in zip(e, w)}
    for M in cubic_ops():
        for v, x in wt.items():
            img = tuple(int(c) for c in M @ np.array(v))
            assert img in wt and wt[img] == pytest.approx(x, rel=1e-14)
    # first moment vanishes; the second, khat e, is isotropic with the virial coefficient
    np.testing.assert_allclose(w @ k, 0.0, atol=1e-13)
    M2 = sigma ** 2 * np.einsum("m,ma,mb->ab", w, k, ef)
    np.testing.assert_allclose(M2, np.eye(3) * 4 * math.pi * sigma ** 3 / 3, rtol=1e-12, atol=1e-9)
    # the fourth-rank tensor sum w khat_a khat_b e_c e_d is isotropic with the
    # continuum coefficient: (4 pi sigma^2 / 15)(d_ab d_cd + d_ac d_bd + d_ad d_bc)
    T = np.einsum("m,ma,mb,mc,md->abcd", w, k, k, ef, ef)
    d = np.eye(3)
    iso = np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)
    np.testing.assert_allclose(T, iso * 4 * math.pi * sigma ** 2 / 15, rtol=0, atol=1e-11 * sigma ** 2)
    # fewer vectors than the full shell (under half of it from sigma 3 on)
    assert len(e) <= 54 and len(e) < len(full) and (sigma < 3 or len(e) * 2 < len(full))


@pytest.mark.parametrize("sigma", SIGMAS + [1.0, 1.5, 2.25])
def test_compact_selection_matches_brute_force(oracle_mod, sigma):
    ref = brute_force_rule(sigma)
    got = oracle_mod.shell_compact(sigma)
    if ref is None:
        assert got is None
        return
    e, w = got
    assert {tuple(v) for v in e} == set(ref)
    for v, x in zip(e, w):
        assert x == pytest.approx(ref[tuple(v)], rel=1e-10)


def test_oracle_refuses_sigma_without_compact_rule(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.Oracle(4, 4, 4, False, 1.5, 1.0, shell_rule="compact")


def _correlate(field, e, weights, shape):
    K = np.zeros(shape)
    for (ex, ey, ez), c in zip(e, weights):
        K[ez % shape[0], ey % shape[1], ex % shape[2]] += c
    return np.real(np.fft.ifftn(np.fft.fftn(field) * np.conj(np.fft.fftn(K))))


@pytest.mark.parametrize("sigma,shape", [(3.0, (7, 8, 9)), (4.0, (9, 8, 10))])
def test_compact_shell_sums_match_fft(oracle_mod, sigma, shape):
    """With g2 = 1 the shell sums are correlations with per-vector weights."""
    rng = np.random.default_rng(23)
    n0 = 0.5 / sigma ** 3
    n = n0 * (1 + 0.1 * (2 * rng.random(shape) - 1))
    u = 1e-3 * rng.standard_normal((3,) + shape)
    nz, ny, nx = shape
    o = oracle_mod.Oracle(nx, ny, nz, False, sigma, 1.0, closure="ONE", shell_rule="compact")
    o.init(n, u)
    _, C, A = o.fields()
    e, w = oracle_mod.shell_compact(sigma)
    k = e / np.linalg.norm(e.astype(float), axis=1)[:, None]
    beta = 2 * sigma ** 2 * math.sqrt(KT / math.pi)
    corr = lambda f, coef: _correlate(f, e, w * coef, shape)
    nu = n[None] * u
    C_ref = np.zeros((3,) + shape)
    for a in range(3):
        C_ref[a] = -KT * sigma ** 2 * corr(n, k[:, a])
        for b in range(3):
            kk = k[:, a] * k[:, b]
            C_ref[a] += beta * (corr(nu[b], kk) - u[b] * corr(n, kk))
    C_ref *= n[None]
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=1e-13 * np.abs(C_ref).max())

    def S(a, b):
        return (corr(nu[a], k[:, b]) - u[a] * corr(n, k[:, b])) + (corr(nu[b], k[:, a]) - u[b] * corr(n, k[:, a]))

    pa = -(KT / 5) * n * sigma ** 2
    A_ref = np.stack([pa * S(0, 0), pa * S(1, 1), pa * S(2, 2), pa * S(0, 1), pa * S(0, 2), pa * S(1, 2)])
    np.testing.assert_allclose(A, A_ref, rtol=0, atol=1e-12 * np.abs(A_ref).max())


def _eos_ratio(oracle_mod, L, sigma, n0, eps=1e-6):
    z = np.arange(L)
    q = 2 * math.pi / L
    n = (n0 * (1 + eps * np.sin(q * z))).reshape(L, 1, 1)
    o = oracle_mod.Oracle(1, 1, L, False, sigma, 1.0, shell_rule="compact")
    o.init(n)
    _, C, _ = o.fields()
    amp = 2.0 / L * np.sum(C[2, :, 0, 0] * np.cos(q * z))
    b = 2 * math.pi * sigma ** 3 / 3
    chi = math.pi * sigma ** 3 * n0 / 6
    dPdn = KT * b * (2 * n0 * g_cs(chi) + n0 ** 2 * dg_cs(chi) * math.pi * sigma ** 3 / 6)
    return amp / (-dPdn * n0 * eps * q)


@pytest.mark.parametrize("sigma,nstar", [(4.0, 0.573), (3.0, 0.4)])
def test_compact_equation_of_state_long_wave(oracle_mod, sigma, nstar):
    """The mean-field force of a long density wave is -grad of the Enskog
    collisional pressure kT b n^2 g2(n), as with the full shell."""
    n0 = nstar / sigma ** 3
    r1 = _eos_ratio(oracle_mod, 128, sigma, n0)
    r2 = _eos_ratio(oracle_mod, 256, sigma, n0)
    assert abs(1 - r2) < abs(1 - r1) / 3.5
    assert abs((4 * r2 - r1) / 3 - 1) < 2e-5


def _decay_rate(oracle_mod, L, sigma, nstar, tau, K, steps=400, skip=100):
    z = np.arange(L)
    q = 2 * math.pi / L
    n = np.full((L, 1, 1), nstar / sigma ** 3)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = 1e-6 * np.sin(q * z)
    o = oracle_mod.Oracle(1, 1, L, False, sigma, tau, k_cross=K, shell_rule="compact")
    o.init(n, u)
    o.step(skip)
    t, a = [], []
    for s in range(steps - skip):
        o.step(1)
        t.append(s)
        a.append(2.0 / L * np.sum(o.moments()[1][0, :, 0, 0] * np.sin(q * z)))
    return -np.polyfit(t, np.log(a), 1)[0]


def test_compact_shear_viscosity_is_the_continuum_value(oracle_mod):
    """Sec. 4 (Eq. treotto with the cross-over term): eta/n = kT (tau - 1/2)
    [1 + K (4 pi / 15) n* g2 ... ] in the continuum; with the compact moments the
    long-wave decay rate of a transverse wave is that closed form,
    r = q^2 [kT (tau-1/2) + (tau-1/2) K kT n g2 4 pi sigma^3 / 15
             + beta g2 n 2 pi sigma^2 / 15],
    up to O(q^2) relative corrections."""
    sigma, nstar, tau = 4.0, 0.573, 1.0
    n0 = nstar / sigma ** 3
    g = g_cs(math.pi * nstar / 6)
    beta = 2 * sigma ** 2 * math.sqrt(KT / math.pi)
    for K in (2.0, 0.0):
        eta_n = (KT * (tau - 0.5) + (tau - 0.5) * K * KT * n0 * g * 4 * math.pi * sigma ** 3 / 15
                 + beta * g * n0 * 2 * math.pi * sigma ** 2 / 15)
        r1 = _decay_rate(oracle_mod, 128, sigma, nstar, tau, K) / (2 * math.pi / 128) ** 2
        assert r1 == pytest.approx(eta_n, rel=5e-3)


def test_compact_conserves_mass_and_momentum(oracle_mod):
    sigma = 4.0
    n0 = synth.reduced_to_density(0.5, sigma)
    n, _ = synth.uniform_with_noise(9, 10, 11, n0, 2e-2, 5, False)
    rng = np.random.default_rng(9)
    u = 1e-3 * rng.standard_normal((3, 11, 10, 9))
    g = (2e-6, -1e-6, 3e-6)
    o = oracle_mod.Oracle(9, 10, 11, False, sigma, 0.9, g, shell_rule="compact")
    o.init(n, u)
    c, _ = oracle_mod.velocities()
    P0 = np.einsum("qzyx,qa->a", o.populations(), c.astype(float))
    mass = o.moments()[0].sum()
    o.step(20)
    P1 = np.einsum("qzyx,qa->a", o.populations(), c.astype(float))
    assert abs(o.moments()[0].sum() - mass) / mass < 1e-13
    scale = np.abs(o.populations()).sum() * 1e-14
    np.testing.assert_allclose(P1 - P0, 20 * mass * np.array(g), rtol=0, atol=scale)
