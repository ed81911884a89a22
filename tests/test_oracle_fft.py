"""Brute-force pin of the shell sums (Sec. 3, Eq. campoc and Eq. campod)
by the convolution theorem.

With the closure g2 = 1 every shell sum is linear in n or n v, hence a
circular cross-correlation with a kernel on the shell vectors, which numpy's
FFT evaluates without any loop over the shell.  At the first step the field
velocity equals the initial velocity (the populations are at equilibrium,
the previous force and tensor are zero), so the expected C and A follow from
the paper's formulas with du = u(r+e) - u(r):
  F^mf_a  = -kT s^2 sum_e w khat_a n(r+e)
  F^vis_a = 2 s^2 sqrt(kT/pi) sum_e w khat_a khat_b n(r+e) du_b
  C = n (F^mf + F^vis)
  A_ab    = -(kT/5) n s^2 sum_e w n(r+e) (khat_b du_a + khat_a du_b)
"""
import itertools
import math

import numpy as np
import pytest

KT = 1.0 / 3.0


def _shell(sigma):
    R = int(math.floor(sigma + 0.5))
    e = [v for v in itertools.product(range(-R, R + 1), repeat=3)
         if (sigma - 0.5) ** 2 < v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= (sigma + 0.5) ** 2]
    e = np.array(e, dtype=float)
    L = np.linalg.norm(e, axis=1)
    w = (4 * math.pi / 3) * sigma / np.sum(e[:, 2] ** 2 / L)
    return e.astype(int), e / L[:, None], w


def _correlate(field, e, weights, shape):
    """sum_e weights[e] * field(r + e) on a periodic (nz, ny, nx) grid."""
    K = np.zeros(shape)
    for (ex, ey, ez), c in zip(e, weights):
        K[ez % shape[0], ey % shape[1], ex % shape[2]] += c
    return np.real(np.fft.ifftn(np.fft.fftn(field) * np.conj(np.fft.fftn(K))))


@pytest.mark.parametrize("sigma,shape", [(3.0, (7, 8, 9)), (4.0, (8, 8, 8))])
def test_shell_sums_match_fft(oracle_mod, sigma, shape):
    rng = np.random.default_rng(17)
    n0 = 0.5 / sigma ** 3
    n = n0 * (1 + 0.1 * (2 * rng.random(shape) - 1))
    u = 1e-3 * rng.standard_normal((3,) + shape)
    nz, ny, nx = shape
    o = oracle_mod.Oracle(nx, ny, nz, False, sigma, 1.0, closure="ONE")
    o.init(n, u)
    nbar, C, A = o.fields()

    e, k, w = _shell(sigma)
    beta = 2 * sigma ** 2 * math.sqrt(KT / math.pi)
    corr = lambda f, coef: _correlate(f, e, w * coef, shape)
    Fmf = np.stack([-KT * sigma ** 2 * corr(n, k[:, a]) for a in range(3)])
    nu = n[None] * u
    Fv = np.zeros((3,) + shape)
    for a in range(3):
        for b in range(3):
            kk = k[:, a] * k[:, b]
            Fv[a] += beta * (corr(nu[b], kk) - u[b] * corr(n, kk))
    C_ref = n[None] * (Fmf + Fv)
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=1e-13 * np.abs(C_ref).max())

    def S(a, b):
        return (corr(nu[a], k[:, b]) - u[a] * corr(n, k[:, b])) + (corr(nu[b], k[:, a]) - u[b] * corr(n, k[:, a]))

    pa = -(KT / 5) * n * sigma ** 2
    A_ref = np.stack([pa * S(0, 0), pa * S(1, 1), pa * S(2, 2), pa * S(0, 1), pa * S(0, 2), pa * S(1, 2)])
    np.testing.assert_allclose(A, A_ref, rtol=0, atol=1e-12 * np.abs(A_ref).max())

    # smeared density: ball mean, by the same convolution
    R = int(math.floor(sigma / 2))
    b = [v for v in itertools.product(range(-R, R + 1), repeat=3) if v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= sigma ** 2 / 4]
    nbar_ref = _correlate(n, np.array(b), np.full(len(b), 1.0 / len(b)), shape)
    np.testing.assert_allclose(nbar, nbar_ref, rtol=1e-13)
