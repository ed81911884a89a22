"""Viscosity sweeps of Sec. 5, run on the GPU path.

- Pore viscosity (the experiment behind Fig. 2): plane Poiseuille flow of the
  hard-sphere fluid between two smooth walls for a range of slab widths, each
  run to its steady state through the serving loop; the effective viscosity
  eta_eff = <n> g_x H^2 / (12 <u_x>) (H = nz - 2 the hydrodynamic width,
  averages over fluid nodes; the paper's "effective slab width" W - sigma is
  H) normalised by the bulk shear viscosity at the pore's mean density.
- Bulk viscosity (the experiment behind Fig. 1): the decay rate r of a
  transverse wave of wavenumber q in a periodic box gives eta = n r / q^2, with
  and without the cross-over term (K = 2 and 0).

The bulk shear viscosity in closed form is the long-wave limit of that decay
under the same discrete equations (Sec. 4, Eq. treotto, with the lattice shell
sums in place of the angular integrals):
    eta / n = kT (tau - 1/2)                                     kinetic
            + (tau - 1/2) K kT n g2 (4 pi sigma^3 / 15)          cross-over (A-term)
            + (beta / 2) g2 n sum_e w_e khat_x^2 e_z^2           collisional (F^viscous)
with beta = 2 sigma^2 sqrt(kT / pi), g2 the Carnahan-Starling contact value at
the density and w_e the weights of the library's contact shell (uniform for
the full shell; for the compact shell the sum is 4 pi sigma^2 / 15, the
continuum value).  Every sweep takes the shell rule ("full" or "compact").
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import synth
from . import wdlb as w

KT = 1.0 / 3.0


def contact_value(chi: float) -> float:
    """Carnahan-Starling g2 at packing fraction chi."""
    return (1.0 - 0.5 * chi) / (1.0 - chi) ** 3


def bulk_shear_viscosity(n: float, sigma: float, tau: float, k_cross: float = 2.0,
                         shell_rule: str = "full") -> float:
    """Dynamic shear viscosity of the uniform fluid of density n (long-wave limit
    of the discrete equations), in lattice units."""
    e, wshell = w.wdlb_shell_table(sigma, shell_rule)
    e = e.astype(np.float64)
    khat = e / np.linalg.norm(e, axis=1)[:, None]
    g2 = contact_value(math.pi * sigma ** 3 * n / 6.0)
    beta = 2.0 * sigma ** 2 * math.sqrt(KT / math.pi)
    kinetic = KT * (tau - 0.5)
    cross = (tau - 0.5) * k_cross * KT * n * g2 * (4.0 * math.pi * sigma ** 3 / 15.0)
    collisional = 0.5 * beta * g2 * n * float(np.sum(wshell * khat[:, 0] ** 2 * e[:, 2] ** 2))
    return n * (kinetic + cross + collisional)


def pore_viscosity_sweep(chi: float, widths, sigma: float = 4.0, tau: float = 1.0, gx: float = 1e-6,
                         nxy: int = 8, tol: float = 1e-8, max_steps: int = 2_000_000, storage: str = "f32",
                         budget_bytes: int = 8 << 30, timeout_s: float = 1800.0, shell_rule: str = "full"):
    """Steady slit Poiseuille flow at packing fraction chi for every hydrodynamic
    width H in `widths` (lattice units; nz = H + 2), uniform initial density,
    cross-section nxy x nxy (the state stays uniform in x and y).  Returns one
    dict per width with H, steps, mean density, eta_eff, eta_bulk and their
    ratio, in the order of `widths`."""
    n0 = synth.packing_to_density(chi, sigma)
    srv = w.wdlb_server_create(budget_bytes, max_active=max(1, len(widths)), check_every=100, storage=storage,
                               shell_rule=shell_rule)
    ids = {}
    try:
        for H in widths:
            nz = int(H) + 2
            n = np.full((nz, nxy, nxy), n0)
            n[0] = n[-1] = 0.0
            rid = w.wdlb_server_submit(srv, (nxy, nxy, nz), sigma, True, tau, (gx, 0.0, 0.0), n, tol=tol,
                                       max_steps=max_steps)
            ids[rid] = int(H)
        results = {}
        t0 = time.time()
        while len(results) < len(ids) and time.time() - t0 < timeout_s:
            for r in w.wdlb_server_poll(srv):
                results[ids[r["id"]]] = r
            time.sleep(0.01)
    finally:
        w.wdlb_server_destroy(srv)
    out = []
    for H in widths:
        r = results.get(int(H))
        if r is None or r["status"] != 0:
            out.append({"H": int(H), "status": None if r is None else r["status"]})
            continue
        st = r["stats"]
        eta_b = bulk_shear_viscosity(st["mean_n"], sigma, tau, shell_rule=shell_rule)
        out.append({"H": int(H), "status": 0, "steps": r["steps"], "mean_n": st["mean_n"],
                    "eta_eff": st["eta_eff"], "eta_bulk": eta_b, "ratio": st["eta_eff"] / eta_b,
                    "seconds": r["finish_s"] - r["start_s"]})
    return out


def bulk_viscosity_sweep(chis, sigma: float = 8.0, tau: float = 1.0, k_values=(2.0, 0.0), L: int = 256,
                         nxy: int = 8, amplitude: float = 1e-6, storage: str = "f32", shell_rule: str = "full"):
    """Bulk shear viscosity against packing fraction (Sec. 5, the experiment
    behind Fig. 1): a uniform fluid at rest is perturbed by a transverse wave
    u_x = a sin(2 pi z / L) on an nxy x nxy x L periodic box, and its decay
    rate r gives eta = n r / q^2, q = 2 pi / L.  For every packing fraction and
    every K of the A-term (k_values: with and without the cross-over term).
    The amplitude is fitted over one e-fold of decay after a tenth of it.
    Returns dicts with chi, K, n, eta (measured), eta_theory (the long-wave
    closed form) and steps."""
    q = 2.0 * math.pi / L
    z = np.arange(L)
    sz = np.sin(q * z)
    out = []
    for chi in chis:
        n0 = synth.packing_to_density(chi, sigma)
        for K in k_values:
            eta_th = bulk_shear_viscosity(n0, sigma, tau, K, shell_rule)
            rate_th = eta_th / n0 * q * q
            span = int(math.ceil(1.0 / rate_th))               # one e-fold
            every = max(1, span // 8)
            n = np.full((L, nxy, nxy), n0)
            u = np.zeros((3, L, nxy, nxy))
            u[0] = amplitude * sz[:, None, None]
            ctx = w.wdlb_create((nxy, nxy, L), sigma, False, tau, (0.0, 0.0, 0.0), storage=storage,
                                k_cross=K, shell_rule=shell_rule)
            w.wdlb_init_fields(ctx, n, u)
            w.wdlb_step(ctx, span // 10)
            t, a = [], []
            for k in range(9):
                if k:
                    w.wdlb_step(ctx, every)
                t.append(span // 10 + k * every)
                ux = w.wdlb_moments(ctx)[1][0].mean(axis=(1, 2))
                a.append(2.0 / L * float(np.sum(ux * sz)))
            w.wdlb_destroy(ctx)
            rate = -np.polyfit(t, np.log(a), 1)[0]
            out.append({"chi": chi, "K": K, "n": n0, "eta": n0 * rate / (q * q), "eta_theory": eta_th,
                        "steps": t[-1]})
    return out
