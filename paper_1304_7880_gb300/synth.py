"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.  This module holds none of the method's arithmetic: it only
draws noise and lays out initial density and velocity fields.

Noise: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to (seed, node index), mapped to a double in
[0, 1) from its top 53 bits.  Relative noise: n = n0 * (1 + a * (2U - 1)).

Layout: node index i = x + nx*(y + ny*z), numpy shape (nz, ny, nx); velocity
(3, nz, ny, nx).  With walls, planes z = 0 and z = nz-1 are solid (n = 0).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state seed + (idx + 1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def reduced_to_density(n_star: float, sigma: float) -> float:
    """n from the reduced density n* = n sigma^3."""
    return n_star / sigma ** 3


def packing_to_density(chi: float, sigma: float) -> float:
    """n from the packing fraction chi = pi n sigma^3 / 6."""
    return 6.0 * chi / (math.pi * sigma ** 3)


def uniform_with_noise(nx, ny, nz, n0, amp, seed, walls):
    """Uniform density n0 with seeded relative noise of amplitude amp, u = 0."""
    U = uniform01(seed, nx * ny * nz).reshape(nz, ny, nx)
    n = n0 * (1.0 + amp * (2.0 * U - 1.0))
    if walls:
        n[0] = 0.0
        n[-1] = 0.0
    u = np.zeros((3, nz, ny, nx))
    return n, u


def shear_wave(nx, ny, nz, n0, amp_noise, u0, seed, walls=False):
    """Transverse shear wave u_x = u0 sin(2 pi z / nz) on a noisy uniform density."""
    n, u = uniform_with_noise(nx, ny, nz, n0, amp_noise, seed, walls)
    z = np.arange(nz, dtype=np.float64)
    u[0] = (u0 * np.sin(2.0 * math.pi * z / nz))[:, None, None] * np.ones((nz, ny, nx))
    return n, u


# Workloads (names state what they are; sizes follow the configuration list).
def slit_8x8x41(seed: int = 1):
    """Plain slit: 8x8x41, walls z=0,40, sigma=4, n*=0.5, +-1e-3 noise, tau=1, g_x=1e-6."""
    sigma = 4.0
    n0 = reduced_to_density(0.5, sigma)
    n, u = uniform_with_noise(8, 8, 41, n0, 1e-3, seed, True)
    params = dict(nx=8, ny=8, nz=41, walls=True, sigma=sigma, tau=1.0, g=(1e-6, 0.0, 0.0))
    return params, n, u


def bulk_shear_128(seed: int = 2, L: int = 128, sigma: float = 4.0):
    """Bulk periodic box L^3, sigma (default 4), packing fraction 0.3, shear wave 1e-4, noise 1e-4."""
    sigma = float(sigma)
    n0 = packing_to_density(0.3, sigma)
    n, u = shear_wave(L, L, L, n0, 1e-4, 1e-4, seed)
    params = dict(nx=L, ny=L, nz=L, walls=False, sigma=sigma, tau=1.0, g=(0.0, 0.0, 0.0))
    return params, n, u


def slit_poiseuille(nx, ny, nz, n_star, sigma, tau, gx, seed, amp=1e-3):
    """Slit Poiseuille request: walls at z=0 and z=nz-1, body force g_x."""
    n0 = reduced_to_density(n_star, sigma)
    n, u = uniform_with_noise(nx, ny, nz, n0, amp, seed, True)
    params = dict(nx=nx, ny=ny, nz=nz, walls=True, sigma=float(sigma), tau=float(tau), g=(float(gx), 0.0, 0.0))
    return params, n, u


# Highest reduced density drawn for slit pores.  Densities up to n* = 0.8
# exceed the scheme's stability: its uniform fluid is linearly unstable above
# n* ~ 0.71 at sigma 4, and in slits the dense contact layer (n* ~ 1.5 at
# contact) turns unstable in the wall plane first: wide slits hold to n* ~ 0.61
# (sigma 3), 0.575 (sigma 4) and 0.59 (sigma 6).
SLIT_N_STAR_MAX = 0.57


def batched_pores(count: int = 64, seed: int = 4, sigma: float = 4.0, nxy: int = 32,
                  n_star_max: float = SLIT_N_STAR_MAX):
    """Batch of slit pores: H uniform in [3 sigma, 30 sigma] (nz = H + 1),
    n* uniform in [0.1, n_star_max], g_x log-uniform in [1e-7, 1e-5], tau = 1."""
    U = uniform01(seed, 3 * count).reshape(count, 3)
    out = []
    for p in range(count):
        H = int(round(3 * sigma + U[p, 0] * (27 * sigma)))
        nz = H + 1
        n_star = 0.1 + (n_star_max - 0.1) * U[p, 1]
        gx = 10.0 ** (-7.0 + 2.0 * U[p, 2])
        out.append(slit_poiseuille(nxy, nxy, nz, n_star, sigma, 1.0, gx, seed * 1000 + p))
    return out


def serving_requests(rate: float, window_s: float, seed: int = 5, n_star_max: float = SLIT_N_STAR_MAX,
                     ln_sigma: float = 0.5):
    """Poisson arrivals (mean rate per second) over window_s seconds of slit
    Poiseuille requests: sigma in {3, 4, 6}; H/sigma lognormal with median 10
    and log-standard deviation ln_sigma, clipped to [3, 60]; nx = ny uniform in
    16..64; n* uniform in [0.1, n_star_max]; g_x log-uniform in [1e-7, 1e-5];
    tau = 1.  Returns (arrival_time, params, seed) tuples; slit_poiseuille with
    those parameters and seed makes the fields."""
    out = []
    t = 0.0
    k = 0
    while True:
        U = uniform01(seed, 8, offset=8 * k)
        t += -math.log(1.0 - U[0]) / rate
        if t > window_s:
            break
        sigma = (3.0, 4.0, 6.0)[min(2, int(U[1] * 3))]
        # Box-Muller normal from two uniforms
        z = math.sqrt(-2.0 * math.log(1.0 - U[2])) * math.cos(2.0 * math.pi * U[3])
        h = min(60.0, max(3.0, 10.0 * math.exp(ln_sigma * z)))
        nz = int(round(h * sigma)) + 1
        nxy = 16 + min(48, int(U[4] * 49))
        n_star = 0.1 + (n_star_max - 0.1) * U[5]
        gx = 10.0 ** (-7.0 + 2.0 * U[6])
        out.append((t, dict(nx=nxy, ny=nxy, nz=nz, n_star=n_star, sigma=sigma, tau=1.0, gx=gx), seed * 100000 + k))
        k += 1
    return out
