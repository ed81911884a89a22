"""Linear response of the discrete WDLB time step around a uniform fluid at rest
(test infrastructure: an independent derivation that the oracle must match).

On a periodic lattice a small perturbation proportional to exp(i k.r) evolves,
to first order in its amplitude, by one fixed linear map per time step.  This
module builds that map in Fourier space, directly from the definitions of the
scheme, with numpy: the moments (Sec. 2, Eq. colonna), the smeared density
over the lattice ball (Sec. 3), the fields C = n (F^mf + F^viscous) and A of
Eq. campoc and Eq. campod summed over the contact shell, the field-velocity
predictor of the explicit trapezoidal rule (reading R7 below), the collision
with second-order forcing and the A-term source (Eq. SMDB, Eq. eq:dufty2 with
the factor K of Eq. extrapressure), and streaming.  It shares no code with the
oracle: tables and closures are rebuilt here from their rules.

Readings (the same ones the oracle states):
  R1  g2 of the homogeneous fluid: Carnahan-Starling, Percus-Yevick or one.
  R2  g2(r, r+e) at chi of the mean of the two ends' smeared densities.
  R3  smeared density = mean of n over the ball |b|^2 <= (sigma/2)^2.
  R4  shell (sigma-1/2)^2 < |e|^2 <= (sigma+1/2)^2, khat = e/|e|, uniform
      weight w with sigma^2 sum w khat_z e_z = 4 pi sigma^3 / 3.
  R6  k_B T = c_s^2 = 1/3.
  R7  u = (j + F/2)/n, (1 - omega/2) on every source; the fields take the
      predictor v: (1 + H) v = j/n + g/2 + C_prev/(2n) + H v_prev with
      H = kappa beta t_prev / 6, kappa = 2, beta = 2 sigma^2 sqrt(kT/pi),
      t = sum_e w g2 n(r+e); at the first step t_prev = 0 and C_prev = 0.

Linearisation about n = n0, u = 0 (g = 0).  With E(e) = exp(i k.e) and
B(k) = mean over the ball of exp(i k.b):
  dn = sum_q a_q,  dj = sum_q a_q c_q
  dv = (dj/n0 + dC_prev/(2 n0) + H dv_prev) / (1 + H)
  dC = n0 [-kT sigma^2 (g0 + n0 chi_n g0' B/2) dn sum_e w khat E(e)
           + beta g0 n0 sum_e w khat (khat.dv) (E(e) - 1)]
  dA_ab = -(kT/5) sigma^2 n0 g0 n0 sum_e w (E(e) - 1) (khat_b dv_a + khat_a dv_b)
  du = (dj + dC/2)/n0,  dfeq_q = w_q (dn + n0 c_q.du / kT)
  dPhi_q = w_q c_q.dC / kT,  dS_q = K w_q c_q.(dA - tr dA/3).c_q / (2 kT^2)
  df*_q = a_q - omega (a_q - dfeq_q) + (1 - omega/2) (dPhi_q + dS_q)
  a'_q = exp(-i k.c_q) df*_q               (f(r, t+1) = f*(r - c, t))
(chi_n = pi sigma^3 / 6, g0 = g2(chi_n n0), g0' its derivative in chi.)  The
terms that multiply the background's zero velocity or zero force, and the
change of H with t, drop out at first order.

State vector X = (a_0..a_18, v_prev (3), C_prev (3)), complex.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KT = 1.0 / 3.0
KAPPA = 2.0


def d3q19():
    c = [(0, 0, 0)]
    c += [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, v)) == 1]
    c += [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, v)) == 2]
    c = np.array(c, float)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return c, w


def shell_full(sigma):
    """Contact shell of reading R4 and its uniform weight."""
    R = int(math.floor(sigma + 0.5))
    e = np.array([v for v in itertools.product(range(-R, R + 1), repeat=3)
                  if (sigma - 0.5) ** 2 < v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= (sigma + 0.5) ** 2], float)
    L = np.linalg.norm(e, axis=1)
    w = (4 * math.pi / 3) * sigma / np.sum(e[:, 2] ** 2 / L)
    return e, np.full(len(e), w)


def ball(sigma):
    R = int(math.floor(sigma / 2))
    return np.array([v for v in itertools.product(range(-R, R + 1), repeat=3)
                     if 4 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) <= sigma * sigma], float)


def closure(kind, chi):
    """g2 at contact and its derivative in chi (Carnahan-Starling, Percus-Yevick, one)."""
    s = 1.0 - chi
    if kind == "CS":
        return (1 - chi / 2) / s ** 3, (2.5 - chi) / s ** 4
    if kind == "PY":
        return (1 + chi / 2) / s ** 2, (2.5 + chi / 2) / s ** 3
    return 1.0, 0.0


class LinearScheme:
    """One-step linear map of the scheme about a uniform fluid n0 at rest."""

    def __init__(self, sigma, n0, tau, K=2.0, kind="CS", shell=None, interactions=True):
        self.sigma, self.n0, self.tau, self.K = float(sigma), float(n0), float(tau), float(K)
        self.c, self.w = d3q19()
        self.e, self.we = shell if shell is not None else shell_full(sigma)
        self.e = np.asarray(self.e, float)
        self.we = np.asarray(self.we, float)
        self.kh = self.e / np.linalg.norm(self.e, axis=1)[:, None]
        self.b = ball(sigma)
        self.chi_n = math.pi * sigma ** 3 / 6
        self.g0, self.dg0 = closure(kind, self.chi_n * n0)
        self.beta = 2 * sigma ** 2 * math.sqrt(KT / math.pi)
        self.inter = bool(interactions)
        t0 = float(np.sum(self.we)) * self.g0 * n0 if self.inter else 0.0
        self.H0 = KAPPA * self.beta * t0 / 6

    def predictor(self, H):
        """Rows giving dv from X."""
        V = np.zeros((3, 25), complex)
        V[:, :19] = self.c.T / self.n0
        V[:, 19:22] = H * np.eye(3)
        V[:, 22:25] = np.eye(3) / (2 * self.n0)
        return V / (1 + H)

    def matrix(self, k, H):
        k = np.asarray(k, float)
        n0, s2 = self.n0, self.sigma ** 2
        E = np.exp(1j * self.e @ k)
        Bk = np.mean(np.exp(1j * self.b @ k))
        Mn = np.zeros(25, complex)
        Mn[:19] = 1.0
        Mj = np.zeros((3, 25), complex)
        Mj[:, :19] = self.c.T
        V = self.predictor(H)
        if self.inter:
            G = (self.we * E) @ self.kh                                  # sum w khat E
            Gv = (self.we * (E - 1)) @ self.kh                           # sum w khat (E - 1)
            Tv = np.einsum("m,ma,mb->ab", self.we * (E - 1), self.kh, self.kh)
            Cm = n0 * (-KT * s2) * (self.g0 + 0.5 * n0 * self.chi_n * self.dg0 * Bk) * np.outer(G, Mn)
            Cm = Cm + n0 * self.beta * self.g0 * n0 * (Tv @ V)
            pa = -(KT / 5) * s2 * n0 * self.g0 * n0                   # dA = pa (dv Gv^T + Gv dv^T)
        else:
            Cm = np.zeros((3, 25), complex)
            Gv = np.zeros(3, complex)
            pa = 0.0
        U = (Mj + 0.5 * Cm) / n0
        omega = 1.0 / self.tau
        rows = []
        for q in range(19):
            cq, wq = self.c[q], self.w[q]
            feq = wq * (Mn + n0 * (cq @ U) / KT)
            phi = wq * (cq @ Cm) / KT
            # c.A.c = 2 pa (c.dv)(c.Gv); tr A = 2 pa (Gv.dv)
            cAc = 2 * pa * ((cq @ Gv) * (cq @ V) - (cq @ cq) / 3 * (Gv @ V))
            sa = self.K * wq / (2 * KT * KT) * cAc if self.inter else 0.0 * cAc
            ea = np.zeros(25, complex)
            ea[q] = 1.0
            post = ea - omega * (ea - feq) + (1 - 0.5 * omega) * (phi + sa)
            rows.append(np.exp(-1j * (cq @ k)) * post)
        return np.vstack([np.array(rows), V, Cm])

    def initial_state(self, dn, du):
        """Oracle initialisation: f = feq(n, u) to first order, v_prev = u, C_prev = 0."""
        X = np.zeros(25, complex)
        X[:19] = self.w * (dn + self.n0 * (self.c @ np.asarray(du)) / KT)
        X[19:22] = du
        return X

    def readout(self, X):
        """Density and field-velocity amplitudes of the state (t_prev at its background)."""
        return np.sum(X[:19]), self.predictor(self.H0) @ X

    def evolve(self, k, dn, du, steps):
        """Amplitudes (dn, dv) after each of `steps` time steps from the oracle's
        initial state: the first step has H = 0 (t_prev = 0)."""
        X = self.initial_state(dn, du)
        M1 = self.matrix(k, 0.0)
        M = self.matrix(k, self.H0)
        out = []
        for s in range(steps):
            X = (M1 if s == 0 else M) @ X
            out.append(self.readout(X))
        return out

    def spectral_radius(self, k):
        return float(np.max(np.abs(np.linalg.eigvals(self.matrix(k, self.H0)))))


def max_growth(sigma, n0, tau, K=2.0, kind="CS", shell=None, qs=None):
    """Largest |eigenvalue| of the steady map over wave vectors along the
    100, 110 and 111 directions (q in (0, pi]), with the wave vector that gives it."""
    ls = LinearScheme(sigma, n0, tau, K, kind, shell)
    if qs is None:
        qs = np.linspace(0.02, math.pi, 160)
    best, kbest = 0.0, None
    for d in (np.array([0, 0, 1.0]), np.array([0, 1.0, 1.0]), np.array([1.0, 1.0, 1.0])):
        for q in qs:
            k = q * d
            r = ls.spectral_radius(k)
            if r > best:
                best, kbest = r, k
    return best, kbest
