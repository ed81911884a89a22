"""FP64 CPU oracle of the WDLB time step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and this
package imports nothing from the product package: the two share no code, header,
table or constant.  The arithmetic lives in ``wdlb_oracle.c`` (plain C, double
precision, single thread); this module only loads it with ctypes and marshals
numpy arrays.  ``pore_average`` restates the pore-averaged quantities with plain
numpy sums in FP64.

Array layout: node index ``i = x + nx*(y + ny*z)``, i.e. numpy C order
``(nz, ny, nx)``; vectors are ``(3, nz, ny, nx)``, A is ``(6, nz, ny, nx)`` in
the order xx, yy, zz, xy, xz, yz.

Every function below that has a counterpart in the paper names it:
Sec. 2 (Model), Sec. 3 (Hard sphere model), Sec. 5 (Numerical results).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wdlb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libwdlb_oracle.so")
_lib = None

CLOSURES = {"CS": 0, "PY": 1, "ONE": 2}
OMEGA_MODES = {"const": 0, "nbar": 1}
SHELL_RULES = {"full": 0, "compact": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    lib.wo_create.restype = P
    lib.wo_create.argtypes = [I, I, I, I, D, D, D, D, D, I, I, D, D, I, I]
    lib.wo_destroy.argtypes = [P]
    lib.wo_init.argtypes = [P, P, P]
    lib.wo_step.argtypes = [P, L]
    lib.wo_step.restype = I
    lib.wo_moments.argtypes = [P, P, P]
    lib.wo_fields.argtypes = [P, P, P, P]
    lib.wo_thermal_fields.argtypes = [P, P, P, P, P]
    lib.wo_get_populations.argtypes = [P, P]
    lib.wo_set_populations.argtypes = [P, P]
    lib.wo_get_cprev.argtypes = [P, P]
    lib.wo_set_cprev.argtypes = [P, P]
    lib.wo_steps.argtypes = [P]
    lib.wo_steps.restype = L
    lib.wo_unstable.argtypes = [P]
    lib.wo_unstable.restype = I
    lib.wo_velocities.argtypes = [P, P]
    lib.wo_velocities.restype = I
    lib.wo_ball.argtypes = [D, P, I]
    lib.wo_ball.restype = I
    lib.wo_shell.argtypes = [D, P, I, P]
    lib.wo_shell.restype = I
    lib.wo_shell_compact.argtypes = [D, P, P, I]
    lib.wo_shell_compact.restype = I
    lib.wo_closure.argtypes = [I, D]
    lib.wo_closure.restype = D
    lib.wo_collide_node.argtypes = [P, P, P, D, D, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def velocities():
    """D3Q19 velocity set and weights (Sec. 5)."""
    lib = _load()
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib.wo_velocities(_ptr(c), _ptr(w))
    return c, w


def ball(sigma: float) -> np.ndarray:
    """Lattice ball of the smeared density (Sec. 3)."""
    lib = _load()
    m = lib.wo_ball(float(sigma), None, 0)
    b = np.zeros((m, 3), dtype=np.int32)
    lib.wo_ball(float(sigma), _ptr(b), m)
    return b


def shell(sigma: float):
    """Contact shell vectors and their uniform weight (Eq. campoc's integral)."""
    lib = _load()
    w = ctypes.c_double()
    m = lib.wo_shell(float(sigma), None, 0, ctypes.byref(w))
    e = np.zeros((m, 3), dtype=np.int32)
    lib.wo_shell(float(sigma), _ptr(e), m, ctypes.byref(w))
    return e, w.value


def shell_compact(sigma: float):
    """Compact contact shell (a quadrature of this library; the paper's
    integral over khat, Eq. campoc, with two or three cubic orbits of the shell
    and one weight per orbit): vectors (m, 3) and weights (m,), or None when
    no such rule exists at this sigma."""
    lib = _load()
    m = lib.wo_shell_compact(float(sigma), None, None, 0)
    if m == 0:
        return None
    e = np.zeros((m, 3), dtype=np.int32)
    w = np.zeros(m)
    lib.wo_shell_compact(float(sigma), _ptr(e), _ptr(w), m)
    return e, w


def closure(kind: str, chi: float) -> float:
    """Homogeneous contact value g2(sigma+) at packing fraction chi (Sec. 3)."""
    return _load().wo_closure(CLOSURES[kind], float(chi))


def collide_node(fin, F, A6, omega: float, k_cross: float) -> np.ndarray:
    """One-node collision of Sec. 5 step 3 (Eq. SMDB with Eq. eq:dufty2)."""
    lib = _load()
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    A6 = np.ascontiguousarray(A6, dtype=np.float64)
    out = np.zeros(19)
    lib.wo_collide_node(_ptr(fin), _ptr(F), _ptr(A6), float(omega), float(k_cross), _ptr(out))
    return out


class Oracle:
    """One lattice (bulk box or slit between walls at z = 0 and z = nz-1)."""

    def __init__(self, nx, ny, nz, walls, sigma, tau, g=(0.0, 0.0, 0.0), closure="CS",
                 omega_mode="const", k_cross=2.0, n_ref=0.0, interactions=True, shell_rule="full"):
        self.lib = _load()
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        self.walls = bool(walls)
        self.g = tuple(float(v) for v in g)
        self.sigma = float(sigma)
        self.h = self.lib.wo_create(int(nx), int(ny), int(nz), int(bool(walls)), float(sigma), float(tau),
                                    self.g[0], self.g[1], self.g[2], CLOSURES[closure],
                                    OMEGA_MODES[omega_mode], float(k_cross), float(n_ref),
                                    int(bool(interactions)), SHELL_RULES[shell_rule])
        if not self.h:
            raise ValueError("oracle: invalid lattice parameters")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.wo_destroy(self.h)
            self.h = None

    def init(self, n, u=None):
        n = np.ascontiguousarray(n, dtype=np.float64).reshape(self.shape)
        if u is None:
            u = np.zeros((3,) + self.shape)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape((3,) + self.shape)
        self.lib.wo_init(self.h, _ptr(n), _ptr(u))

    def step(self, nsteps: int = 1) -> int:
        return self.lib.wo_step(self.h, int(nsteps))

    @property
    def steps(self) -> int:
        return self.lib.wo_steps(self.h)

    @property
    def unstable(self) -> bool:
        return bool(self.lib.wo_unstable(self.h))

    def moments(self):
        n = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        self.lib.wo_moments(self.h, _ptr(n), _ptr(u))
        return n, u

    def fields(self):
        nbar = np.zeros(self.shape)
        C = np.zeros((3,) + self.shape)
        A = np.zeros((6,) + self.shape)
        self.lib.wo_fields(self.h, _ptr(nbar), _ptr(C), _ptr(A))
        return nbar, C, A

    def thermal_fields(self, T):
        """Energy-equation fields of Sec. 3 on a prescribed temperature field T
        (k_B T per node, lattice units): Q (Eq. campob1), B (Eq. campos) and
        the thermal force F^T (Eq. thermalforce), on the current populations."""
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.shape)
        Qf = np.zeros(self.shape)
        B = np.zeros((3,) + self.shape)
        FT = np.zeros((3,) + self.shape)
        self.lib.wo_thermal_fields(self.h, _ptr(T), _ptr(Qf), _ptr(B), _ptr(FT))
        return Qf, B, FT

    def populations(self) -> np.ndarray:
        f = np.zeros((19,) + self.shape)
        self.lib.wo_get_populations(self.h, _ptr(f))
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((19,) + self.shape)
        self.lib.wo_set_populations(self.h, _ptr(f))

    def cprev(self) -> np.ndarray:
        c = np.zeros((3,) + self.shape)
        self.lib.wo_get_cprev(self.h, _ptr(c))
        return c

    def set_cprev(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64).reshape((3,) + self.shape)
        self.lib.wo_set_cprev(self.h, _ptr(c))


def pore_average(n, u, walls: bool, gx: float):
    """Pore-averaged quantities (abstract: "pore-averaged properties").

    mean_n, mean_ux over fluid nodes; flux_x = sum n u_x / (nx ny);
    eta_eff = <n> g_x H^2 / (12 <u_x>) with hydrodynamic width H = nz - 2
    (the mean of a plane Poiseuille profile of viscosity eta), NaN without walls.
    """
    nz, ny, nx = n.shape
    fluid = np.ones(n.shape, dtype=bool)
    if walls:
        fluid[0] = False
        fluid[-1] = False
    nf = n[fluid]
    uxf = u[0][fluid]
    mean_n = float(np.sum(nf) / nf.size)
    mean_ux = float(np.sum(uxf) / uxf.size)
    flux = float(np.sum(nf * uxf) / (nx * ny))
    if walls and mean_ux != 0.0:
        H = nz - 2
        eta = mean_n * gx * H * H / (12.0 * mean_ux)
    else:
        eta = float("nan")
    return {"mean_n": mean_n, "mean_ux": mean_ux, "flux_x": flux, "eta_eff": eta}
