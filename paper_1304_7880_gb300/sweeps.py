"""Pore-viscosity sweep of Sec. 5 (the experiment behind Fig. 2): plane
Poiseuille flow of the hard-sphere fluid between two smooth walls, for a range
of slab widths, each run to its steady state on the GPU through the serving
loop, and the effective viscosity of the pore normalised by the bulk shear
viscosity at the pore's mean density.

- Effective viscosity (pore average): eta_eff = <n> g_x H^2 / (12 <u_x>), with
  H = nz - 2 the hydrodynamic width and averages over fluid nodes
  (wdlb_pore_average).  The paper's "effective slab width" W - sigma is H.
- Bulk shear viscosity: the long-wave limit of the decay of a transverse wave
  under the same discrete equations (Sec. 4, Eq. treotto, with the lattice
  shell sums in place of the angular integrals):
      eta / n = kT (tau - 1/2)                                     kinetic
              + (tau - 1/2) K kT n g2 (4 pi sigma^3 / 15)          cross-over (A-term)
              + (beta / 2) g2 n sum_e w khat_x^2 e_z^2             collisional (F^viscous)
  with beta = 2 sigma^2 sqrt(kT / pi), g2 the Carnahan-Starling contact value
  at the density and w the library's uniform shell weight.
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


def bulk_shear_viscosity(n: float, sigma: float, tau: float, k_cross: float = 2.0) -> float:
    """Dynamic shear viscosity of the uniform fluid of density n (long-wave limit
    of the discrete equations), in lattice units."""
    e, wshell = w.wdlb_stencil(sigma, 1)
    e = e.astype(np.float64)
    khat = e / np.linalg.norm(e, axis=1)[:, None]
    g2 = contact_value(math.pi * sigma ** 3 * n / 6.0)
    beta = 2.0 * sigma ** 2 * math.sqrt(KT / math.pi)
    kinetic = KT * (tau - 0.5)
    cross = (tau - 0.5) * k_cross * KT * n * g2 * (4.0 * math.pi * sigma ** 3 / 15.0)
    collisional = 0.5 * beta * g2 * n * wshell * float(np.sum(khat[:, 0] ** 2 * e[:, 2] ** 2))
    return n * (kinetic + cross + collisional)


def pore_viscosity_sweep(chi: float, widths, sigma: float = 4.0, tau: float = 1.0, gx: float = 1e-6,
                         nxy: int = 8, tol: float = 1e-8, max_steps: int = 2_000_000, storage: str = "f32",
                         budget_bytes: int = 8 << 30, timeout_s: float = 1800.0):
    """Steady slit Poiseuille flow at packing fraction chi for every hydrodynamic
    width H in `widths` (lattice units; nz = H + 2), uniform initial density,
    cross-section nxy x nxy (the state stays uniform in x and y).  Returns one
    dict per width with H, steps, mean density, eta_eff, eta_bulk and their
    ratio, in the order of `widths`."""
    n0 = synth.packing_to_density(chi, sigma)
    srv = w.wdlb_server_create(budget_bytes, max_active=max(1, len(widths)), check_every=100, storage=storage)
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
        eta_b = bulk_shear_viscosity(st["mean_n"], sigma, tau)
        out.append({"H": int(H), "status": 0, "steps": r["steps"], "mean_n": st["mean_n"],
                    "eta_eff": st["eta_eff"], "eta_bulk": eta_b, "ratio": st["eta_eff"] / eta_b,
                    "seconds": r["finish_s"] - r["start_s"]})
    return out
