"""ctypes binding of the WDLB C ABI (``include/wdlb.h``), same names.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libwdlb.so``.  PyTorch supplies the device memory (one workspace tensor per
context, handed to the library) and the CUDA stream.  There is no CPU path: if
the compiled library is missing, loading fails with an error.

Arrays: node index i = x + nx*(y + ny*z), numpy shape (nz, ny, nx); vectors
(3, nz, ny, nx); A (6, nz, ny, nx) in the order xx, yy, zz, xy, xz, yz.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# WDLB_LIBRARY selects another build of the library (the bounds-checked one).
LIB_PATH = os.environ.get("WDLB_LIBRARY") or os.path.join(_HERE, "_build", "libwdlb.so")
_lib = None

WDLB_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_UNSTABLE", 5: "ERR_TIMEOUT",
                6: "ERR_STATE"}
CLOSURES = {"CS": 0, "PY": 1, "ONE": 2}
OMEGA_MODES = {"const": 0, "nbar": 1}
STORAGES = {"f64": 0, "f32": 1, "f16": 2}
SHELL_RULES = {"full": 0, "compact": 1}


class WDLBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class wdlb_lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class wdlb_options(ctypes.Structure):
    _fields_ = [("closure", ctypes.c_int32), ("omega_mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("interactions", ctypes.c_int32), ("k_cross", ctypes.c_double), ("n_ref", ctypes.c_double),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("tile", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("shell_rule", ctypes.c_int32), ("staging", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("collision", ctypes.c_int32)]


STAGINGS = {"auto": 0, "cp_async": 1}
# arithmetic of the collision with FP32 storage: "fp32", or "dw" (double-word
# pairs of floats; lattices with walls)
COLLISIONS = {"fp32": 0, "dw": 1}


class wdlb_pore_desc(ctypes.Structure):
    _fields_ = [("lat", wdlb_lattice), ("sigma", ctypes.c_double), ("walls", ctypes.c_int32),
                ("tau", ctypes.c_double), ("g", ctypes.c_double * 3)]


class wdlb_request(ctypes.Structure):
    _fields_ = [("desc", wdlb_pore_desc), ("n", ctypes.c_void_p), ("u", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("out_n", ctypes.c_void_p), ("out_u", ctypes.c_void_p)]


class wdlb_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active", ctypes.c_int64), ("pool_free", ctypes.c_uint64),
                ("launches", ctypes.c_int64), ("clock_s", ctypes.c_double), ("node_steps", ctypes.c_int64),
                ("gpu_step_s", ctypes.c_double)]


class wdlb_pore_stats(ctypes.Structure):
    _fields_ = [("mean_n", ctypes.c_double), ("mean_ux", ctypes.c_double), ("flux_x", ctypes.c_double),
                ("mass", ctypes.c_double), ("eta_eff", ctypes.c_double), ("residual", ctypes.c_double),
                ("steps", ctypes.c_int64)]


def load_library(path: str = LIB_PATH):
    """Load libwdlb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libwdlb.so not built (%s); run paper_1304_7880_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "wdlb_default_options": (None, [P]),
        "wdlb_workspace_size": (I32, [wdlb_lattice, D, I32, P, P]),
        "wdlb_create": (I32, [wdlb_lattice, D, I32, D, P, P, P]),
        "wdlb_init_fields": (I32, [P, P, P]),
        "wdlb_init_fields_device": (I32, [P, P, P]),
        "wdlb_step": (I32, [P, I64]),
        "wdlb_moments": (I32, [P, P, P]),
        "wdlb_moments_device": (I32, [P, P, P]),
        "wdlb_fields": (I32, [P, P, P, P, P]),
        "wdlb_thermal_fields": (I32, [P, P, P, P, P]),
        "wdlb_get_populations": (I32, [P, P]),
        "wdlb_pore_average": (I32, [P, P]),
        "wdlb_run_steady": (I32, [P, D, I32, I64, P, P]),
        "wdlb_autotune": (I32, [wdlb_lattice, D, I32, P, P, P]),
        "wdlb_state_bytes": (I32, [P, P]),
        "wdlb_save_state": (I32, [P, P, ctypes.c_uint64]),
        "wdlb_load_state": (I32, [P, P, ctypes.c_uint64]),
        "wdlb_tile_info": (I32, [P, P, P]),
        "wdlb_autotune_reset": (None, []),
        "wdlb_velocity_set": (I32, [P, P]),
        "wdlb_stencil": (I32, [D, I32, P, I32, P, P]),
        "wdlb_shell_table": (I32, [D, I32, P, P, I32, P]),
        "wdlb_profile_step": (I32, [P, I64, P]),
        "wdlb_fields_static": (I32, [wdlb_lattice, D, I32, I32, P, P, P, P, P, P]),
        "wdlb_launch_count": (I64, [P]),
        "wdlb_staging_info": (I32, [P, P]),
        "wdlb_last_error": (ctypes.c_char_p, [P]),
        "wdlb_batch_create": (I32, [P, ctypes.c_uint64, I32, P]),
        "wdlb_batch_pore_bytes": (I32, [P, P, P]),
        "wdlb_batch_add": (I32, [P, P, P, P, P]),
        "wdlb_batch_remove": (I32, [P, I32]),
        "wdlb_batch_step": (I32, [P, I64]),
        "wdlb_batch_profile_step": (I32, [P, I64, P]),
        "wdlb_batch_residuals": (I32, [P, I32, P, P]),
        "wdlb_batch_context": (P, [P, I32]),
        "wdlb_batch_active": (I32, [P]),
        "wdlb_batch_free_bytes": (ctypes.c_uint64, [P]),
        "wdlb_batch_launch_count": (I64, [P]),
        "wdlb_batch_last_error": (ctypes.c_char_p, [P]),
        "wdlb_batch_destroy": (None, [P]),
        "wdlb_server_create": (I32, [P, ctypes.c_uint64, I32, I32, P]),
        "wdlb_server_submit": (I32, [P, P, P]),
        "wdlb_server_poll": (I32, [P, P, I32]),
        "wdlb_server_info": (I32, [P, P]),
        "wdlb_server_destroy": (None, [P]),
        "wdlb_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != WDLB_OK:
        lib = load_library()
        msg = lib.wdlb_last_error(ctx.handle if ctx is not None else None)
        raise WDLBError(status, msg.decode() if msg else "")


def _f64(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError("expected %d values, got %d" % (int(np.prod(shape)), a.size))
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """Handle of one lattice plus the torch objects that back it."""

    def __init__(self, handle, shape, workspace, stream, walls, g):
        self.handle = handle
        self.shape = shape          # (nz, ny, nx)
        self.N = int(np.prod(shape))
        self.workspace = workspace  # torch uint8 tensor (device memory)
        self.stream = stream        # torch.cuda.Stream
        self.walls = walls
        self.g = g

    def __del__(self):
        if getattr(self, "handle", None):
            wdlb_destroy(self)


def wdlb_create(lattice, sigma, walls, tau, g=(0.0, 0.0, 0.0), closure="CS", omega_mode="const",
                storage="f32", interactions=True, k_cross=2.0, n_ref=0.0, device=None, tile=-1, autotune=True,
                shell_rule="full", staging="auto", wait_limit=0, collision="fp32"):
    """Create a context; device memory and stream come from PyTorch.  tile: -1
    (autotuner) or a forced tile shape 0, 1, 2 of the tiled shell kernel;
    shell_rule: "full" or "compact" contact-shell quadrature; staging: "auto"
    (TMA tiles where possible) or "cp_async"; wait_limit: polls of the TMA
    tile's wait (0: the library's default); collision: "fp32" or "dw"
    (double-word collision, FP32 storage with walls)."""
    import torch

    lib = load_library()
    nx, ny, nz = (int(v) for v in lattice)
    lat = wdlb_lattice(nx, ny, nz)
    opt = wdlb_options()
    lib.wdlb_default_options(ctypes.byref(opt))
    opt.closure = CLOSURES[closure]
    opt.omega_mode = OMEGA_MODES[omega_mode]
    opt.storage = STORAGES[storage]
    opt.interactions = 1 if interactions else 0
    opt.k_cross = float(k_cross)
    opt.n_ref = float(n_ref)
    opt.tile = int(tile)
    opt.autotune = 1 if autotune else 0
    opt.shell_rule = SHELL_RULES[shell_rule]
    opt.staging = STAGINGS[staging]
    opt.wait_limit = int(wait_limit)
    opt.collision = COLLISIONS[collision]
    walls_i = 1 if walls else 0
    nbytes = ctypes.c_uint64()
    _check(lib.wdlb_workspace_size(lat, float(sigma), walls_i, ctypes.byref(opt), ctypes.byref(nbytes)))
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    stream = torch.cuda.Stream(device=dev)
    opt.workspace = ctypes.c_void_p(aligned)
    opt.workspace_bytes = int(nbytes.value)
    opt.stream = ctypes.c_void_p(stream.cuda_stream)
    gg = (ctypes.c_double * 3)(*[float(v) for v in g])
    handle = ctypes.c_void_p()
    with torch.cuda.device(dev):
        _check(lib.wdlb_create(lat, float(sigma), walls_i, float(tau), gg, ctypes.byref(opt), ctypes.byref(handle)))
    return Context(handle, (nz, ny, nx), workspace, stream, bool(walls), tuple(float(v) for v in g))


def wdlb_init_fields(ctx: Context, n, u=None):
    lib = load_library()
    n = _f64(n, ctx.shape)
    uu = None if u is None else _f64(u, (3,) + ctx.shape)
    _check(lib.wdlb_init_fields(ctx.handle, _ptr(n), None if uu is None else _ptr(uu)), ctx)


def wdlb_init_fields_device(ctx: Context, d_n, d_u=None):
    """d_n, d_u: float64 CUDA tensors (N and 3N values), read on the context stream."""
    lib = load_library()
    _check(lib.wdlb_init_fields_device(ctx.handle, ctypes.c_void_p(d_n.data_ptr()),
                                       None if d_u is None else ctypes.c_void_p(d_u.data_ptr())), ctx)


def wdlb_step(ctx: Context, nsteps: int = 1):
    _check(load_library().wdlb_step(ctx.handle, int(nsteps)), ctx)


def wdlb_moments(ctx: Context, n_out=None, u_out=None):
    """Density and field velocity as numpy arrays (host; synchronous)."""
    lib = load_library()
    n = np.empty(ctx.shape) if n_out is None else n_out
    u = np.empty((3,) + ctx.shape) if u_out is None else u_out
    _check(lib.wdlb_moments(ctx.handle, _ptr(n), _ptr(u)), ctx)
    return n, u


def wdlb_moments_device(ctx: Context, d_n, d_u):
    lib = load_library()
    _check(lib.wdlb_moments_device(ctx.handle, None if d_n is None else ctypes.c_void_p(d_n.data_ptr()),
                                   None if d_u is None else ctypes.c_void_p(d_u.data_ptr())), ctx)


def wdlb_fields(ctx: Context):
    """nbar, C, A, u (trapezoidal velocity) of the current state (host arrays)."""
    lib = load_library()
    nbar = np.empty(ctx.shape)
    C = np.empty((3,) + ctx.shape)
    A = np.empty((6,) + ctx.shape)
    u = np.empty((3,) + ctx.shape)
    _check(lib.wdlb_fields(ctx.handle, _ptr(nbar), _ptr(C), _ptr(A), _ptr(u)), ctx)
    return nbar, C, A, u


def wdlb_thermal_fields(ctx: Context, T):
    """Energy-equation fields of Sec. 3 on a prescribed temperature T (k_B T per
    node, lattice units; shape (nz, ny, nx)): (Q, B, FT) with shapes
    (nz, ny, nx), (3, nz, ny, nx), (3, nz, ny, nx) (Eq. campob1, Eq. campos,
    Eq. thermalforce)."""
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(ctx.shape)
    Qf = np.empty(ctx.shape)
    B = np.empty((3,) + ctx.shape)
    FT = np.empty((3,) + ctx.shape)
    _check(load_library().wdlb_thermal_fields(ctx.handle, _ptr(T), _ptr(Qf), _ptr(B), _ptr(FT)), ctx)
    return Qf, B, FT


def wdlb_get_populations(ctx: Context) -> np.ndarray:
    lib = load_library()
    f = np.empty((19,) + ctx.shape)
    _check(lib.wdlb_get_populations(ctx.handle, _ptr(f)), ctx)
    return f


def wdlb_pore_average(ctx: Context) -> dict:
    lib = load_library()
    st = wdlb_pore_stats()
    _check(lib.wdlb_pore_average(ctx.handle, ctypes.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in wdlb_pore_stats._fields_}


def wdlb_save_state(ctx: Context) -> np.ndarray:
    """Checkpoint of the context's state (an opaque byte array)."""
    lib = load_library()
    nb = ctypes.c_uint64()
    _check(lib.wdlb_state_bytes(ctx.handle, ctypes.byref(nb)), ctx)
    buf = np.zeros(int(nb.value), dtype=np.uint8)
    _check(lib.wdlb_save_state(ctx.handle, _ptr(buf), ctypes.c_uint64(buf.nbytes)), ctx)
    return buf


def wdlb_load_state(ctx: Context, buf: np.ndarray):
    """Restore a checkpoint taken from a context of the same configuration."""
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().wdlb_load_state(ctx.handle, _ptr(buf), ctypes.c_uint64(buf.nbytes)), ctx)


def wdlb_autotune(lattice, sigma, walls, storage="f32", device=None, shell_rule="full", collision="fp32"):
    """Time the tiled shell kernel's shapes for this (storage, sigma, walls, nz,
    shell rule, collision) now and record the fastest; returns (best, [ms per
    step of shapes 0, 1, 2])."""
    import torch

    lib = load_library()
    opt = wdlb_options()
    lib.wdlb_default_options(ctypes.byref(opt))
    opt.storage = STORAGES[storage]
    opt.shell_rule = SHELL_RULES[shell_rule]
    opt.collision = COLLISIONS[collision]
    nx, ny, nz = (int(v) for v in lattice)
    best = ctypes.c_int32()
    ms = (ctypes.c_double * 3)()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        st = lib.wdlb_autotune(wdlb_lattice(nx, ny, nz), float(sigma), 1 if walls else 0, ctypes.byref(opt),
                               ctypes.byref(best), ms)
    if st != WDLB_OK:
        raise WDLBError(st, "wdlb_autotune")
    return best.value, list(ms)


def wdlb_tile_info(ctx: Context):
    """(tiled, tile shape) of the shell kernel the context runs."""
    tiled, tile = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().wdlb_tile_info(ctx.handle, ctypes.byref(tiled), ctypes.byref(tile)), ctx)
    return bool(tiled.value), tile.value


def wdlb_staging_info(ctx: Context) -> bool:
    """True if the context's tiled shell kernel loads interior tiles by TMA."""
    tma = ctypes.c_int32()
    _check(load_library().wdlb_staging_info(ctx.handle, ctypes.byref(tma)), ctx)
    return bool(tma.value)


def wdlb_autotune_reset():
    load_library().wdlb_autotune_reset()


def wdlb_run_steady(ctx: Context, tol: float, check_every: int = 100, max_steps: int = 10 ** 7):
    lib = load_library()
    done = ctypes.c_int64()
    res = ctypes.c_double()
    _check(lib.wdlb_run_steady(ctx.handle, float(tol), int(check_every), int(max_steps), ctypes.byref(done),
                               ctypes.byref(res)), ctx)
    return done.value, res.value


def wdlb_velocity_set():
    lib = load_library()
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    _check(lib.wdlb_velocity_set(_ptr(c), _ptr(w)))
    return c, w


def wdlb_stencil(sigma: float, which: int):
    """which = 0: smeared-density ball; 1: contact shell (vectors, weight)."""
    lib = load_library()
    cnt = ctypes.c_int32()
    w = ctypes.c_double()
    _check(lib.wdlb_stencil(float(sigma), int(which), None, 0, ctypes.byref(cnt), ctypes.byref(w)))
    v = np.zeros((cnt.value, 3), dtype=np.int32)
    _check(lib.wdlb_stencil(float(sigma), int(which), _ptr(v), cnt.value, ctypes.byref(cnt), ctypes.byref(w)))
    return v, w.value


def wdlb_shell_table(sigma: float, rule: str = "full"):
    """Contact shell of a quadrature rule: vectors (m, 3), +e and -e adjacent,
    and the weight of each (m,)."""
    lib = load_library()
    cnt = ctypes.c_int32()
    _check(lib.wdlb_shell_table(float(sigma), SHELL_RULES[rule], None, None, 0, ctypes.byref(cnt)))
    v = np.zeros((cnt.value, 3), dtype=np.int32)
    w = np.zeros(cnt.value)
    _check(lib.wdlb_shell_table(float(sigma), SHELL_RULES[rule], _ptr(v), _ptr(w), cnt.value, ctypes.byref(cnt)))
    return v, w


def wdlb_profile_step(ctx: Context, nsteps: int):
    """Advance nsteps with per-kernel CUDA events; mean ms per launch of
    (moments, smeared density, shell + collide + stream)."""
    ms = (ctypes.c_double * 3)()
    _check(load_library().wdlb_profile_step(ctx.handle, int(nsteps), ms), ctx)
    return tuple(ms)


WDLB_STATIC_MAX_NODES = 262144


def _check_device_tensor(call, name, t, count):
    """A float64 tensor on the current CUDA device, contiguous, of `count`
    elements; WDLBError(ERR_ARG) otherwise."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
          and t.numel() == count)
    if ok and t.device.index != torch.cuda.current_device():
        ok = False
    if not ok:
        desc = ("%s %s on %s, %d elements" % (type(t).__name__, getattr(t, "dtype", "?"), getattr(t, "device", "?"),
                                                getattr(t, "numel", lambda: -1)()))
        raise WDLBError(1, "%s: %s must be a contiguous float64 tensor of %d elements on the current CUDA device "
                           "(got %s)" % (call, name, count, desc))


def wdlb_fields_static(lattice, sigma, walls, closure, d_n, d_u, d_nbar, d_C, d_A, stream=None):
    """Fields (nbar, C, A) of device arrays n, u without any device allocation
    (see include/wdlb.h): torch CUDA tensors of float64, results written into
    d_nbar (may be None), d_C, d_A; enqueued on `stream` (torch.cuda.Stream or
    None for the legacy default stream)."""
    nx, ny, nz = (int(v) for v in lattice)
    N = nx * ny * nz
    # the C side cannot see a buffer's type or size: a wrong one would be
    # read or written past its end, so every tensor is checked here first
    for name, t, count, required in (("n", d_n, N, True), ("u", d_u, 3 * N, True), ("nbar", d_nbar, N, False),
                                     ("C", d_C, 3 * N, True), ("A", d_A, 6 * N, True)):
        if t is None:
            if required:
                raise WDLBError(1, "wdlb_fields_static: %s is required" % name)
            continue
        _check_device_tensor("wdlb_fields_static", name, t, count)
    lib = load_library()
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib.wdlb_fields_static(wdlb_lattice(nx, ny, nz), float(sigma), 1 if walls else 0, CLOSURES[closure],
                                  ptr(d_n), ptr(d_u), ptr(d_nbar), ptr(d_C), ptr(d_A), st))


def wdlb_launch_count(ctx: Context) -> int:
    return int(load_library().wdlb_launch_count(ctx.handle))


def wdlb_last_error(ctx: Context = None) -> str:
    msg = load_library().wdlb_last_error(None if ctx is None else ctx.handle)
    return msg.decode() if msg else ""


def wdlb_destroy(ctx: Context):
    if ctx.handle:
        load_library().wdlb_destroy(ctx.handle)
        ctx.handle = None


# ---- batches of independent lattices -------------------------------------------------

class Batch:
    """Handle of a batch plus the torch pool and stream that back it."""

    def __init__(self, handle, pool, stream, max_pores):
        self.handle = handle
        self.pool = pool
        self.stream = stream
        self.max_pores = max_pores
        self.shapes = {}

    def __del__(self):
        if getattr(self, "handle", None):
            wdlb_batch_destroy(self)


class SlotContext(Context):
    """A batch slot's context (owned by the batch; never destroyed here)."""

    def __del__(self):
        pass


def _bcheck(status, batch=None):
    if status != WDLB_OK:
        msg = load_library().wdlb_batch_last_error(None if batch is None else batch.handle)
        raise WDLBError(status, msg.decode() if msg else "")


def wdlb_batch_create(max_pores, pool_bytes, closure="CS", omega_mode="const", storage="f32", interactions=True,
                      k_cross=2.0, device=None, shell_rule="full", autotune=True, staging="auto",
                      persistent=False, wait_limit=0, collision="fp32"):
    import torch

    lib = load_library()
    opt = wdlb_options()
    lib.wdlb_default_options(ctypes.byref(opt))
    opt.collision = COLLISIONS[collision]
    opt.closure = CLOSURES[closure]
    opt.omega_mode = OMEGA_MODES[omega_mode]
    opt.storage = STORAGES[storage]
    opt.interactions = 1 if interactions else 0
    opt.k_cross = float(k_cross)
    opt.shell_rule = SHELL_RULES[shell_rule]
    opt.autotune = 1 if autotune else 0
    opt.staging = STAGINGS[staging]
    opt.persistent = 1 if persistent else 0
    opt.wait_limit = int(wait_limit)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    pool = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    opt.workspace = ctypes.c_void_p((pool.data_ptr() + 255) & ~255)
    opt.workspace_bytes = int(pool_bytes)
    opt.stream = ctypes.c_void_p(stream.cuda_stream)
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        _bcheck(lib.wdlb_batch_create(ctypes.byref(opt), int(pool_bytes), int(max_pores), ctypes.byref(h)))
    return Batch(h, pool, stream, int(max_pores))


def _desc(lattice, sigma, walls, tau, g):
    nx, ny, nz = (int(v) for v in lattice)
    return wdlb_pore_desc(wdlb_lattice(nx, ny, nz), float(sigma), 1 if walls else 0, float(tau),
                          (ctypes.c_double * 3)(*[float(v) for v in g]))


def wdlb_batch_pore_bytes(batch, lattice, sigma, walls, tau=1.0, g=(0.0, 0.0, 0.0)) -> int:
    d = _desc(lattice, sigma, walls, tau, g)
    nb = ctypes.c_uint64()
    _bcheck(load_library().wdlb_batch_pore_bytes(batch.handle, ctypes.byref(d), ctypes.byref(nb)), batch)
    return nb.value


def wdlb_batch_add(batch, lattice, sigma, walls, tau, g, n, u=None) -> int:
    nx, ny, nz = (int(v) for v in lattice)
    shape = (nz, ny, nx)
    d = _desc(lattice, sigma, walls, tau, g)
    nn = _f64(n, shape)
    uu = None if u is None else _f64(u, (3,) + shape)
    slot = ctypes.c_int32()
    _bcheck(load_library().wdlb_batch_add(batch.handle, ctypes.byref(d), _ptr(nn), None if uu is None else _ptr(uu),
                                          ctypes.byref(slot)), batch)
    batch.shapes[slot.value] = (shape, bool(walls), tuple(float(v) for v in g))
    return slot.value


def wdlb_batch_remove(batch, slot):
    _bcheck(load_library().wdlb_batch_remove(batch.handle, int(slot)), batch)
    batch.shapes.pop(int(slot), None)


def wdlb_batch_step(batch, nsteps=1):
    _bcheck(load_library().wdlb_batch_step(batch.handle, int(nsteps)), batch)


def wdlb_batch_profile_step(batch, nsteps=1):
    """nsteps time steps launched kernel by kernel with CUDA events around each
    phase; returns the average ms per step of (moments, smeared density, shell
    sums + collision + streaming)."""
    ms = (ctypes.c_double * 3)()
    _bcheck(load_library().wdlb_batch_profile_step(batch.handle, int(nsteps), ms), batch)
    return [ms[0], ms[1], ms[2]]


def wdlb_batch_residuals(batch, interval):
    res = np.full(batch.max_pores, np.nan)
    st = np.zeros(batch.max_pores, dtype=np.int32)
    _bcheck(load_library().wdlb_batch_residuals(batch.handle, int(interval), _ptr(res), _ptr(st)), batch)
    return res, st


def wdlb_batch_context(batch, slot) -> SlotContext:
    h = load_library().wdlb_batch_context(batch.handle, int(slot))
    if not h:
        raise WDLBError(1, "empty slot %d" % slot)
    shape, walls, g = batch.shapes[int(slot)]
    return SlotContext(ctypes.c_void_p(h), shape, None, batch.stream, walls, g)


def wdlb_batch_active(batch) -> int:
    return int(load_library().wdlb_batch_active(batch.handle))


def wdlb_batch_free_bytes(batch) -> int:
    return int(load_library().wdlb_batch_free_bytes(batch.handle))


def wdlb_batch_launch_count(batch) -> int:
    return int(load_library().wdlb_batch_launch_count(batch.handle))


def wdlb_batch_destroy(batch):
    if batch.handle:
        load_library().wdlb_batch_destroy(batch.handle)
        batch.handle = None


# ---- serving ---------------------------------------------------------------------------

class wdlb_result(ctypes.Structure):
    pass


class Server:
    def __init__(self, handle, pool, stream):
        self.handle = handle
        self.pool = pool
        self.stream = stream
        self.keep = {}     # id -> host arrays that must outlive the request
        self.nodes = {}    # id -> lattice nodes (for the per-solve log)

    def __del__(self):
        if getattr(self, "handle", None):
            wdlb_server_destroy(self)


def wdlb_server_create(hbm_budget, max_active=256, check_every=100, closure="CS", storage="f32", device=None,
                       shell_rule="full", collision="fp32"):
    """Serving loop (native worker thread) over a batch whose pool is a torch tensor."""
    import torch

    lib = load_library()
    opt = wdlb_options()
    lib.wdlb_default_options(ctypes.byref(opt))
    opt.collision = COLLISIONS[collision]
    opt.closure = CLOSURES[closure]
    opt.storage = STORAGES[storage]
    opt.shell_rule = SHELL_RULES[shell_rule]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    pool = torch.empty(int(hbm_budget) + 256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    opt.workspace = ctypes.c_void_p((pool.data_ptr() + 255) & ~255)
    opt.workspace_bytes = int(hbm_budget)
    opt.stream = ctypes.c_void_p(stream.cuda_stream)
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        st = lib.wdlb_server_create(ctypes.byref(opt), int(hbm_budget), int(max_active), int(check_every),
                                    ctypes.byref(h))
    if st != WDLB_OK:
        raise WDLBError(st, "wdlb_server_create")
    return Server(h, pool, stream)


def wdlb_server_submit(server, lattice, sigma, walls, tau, g, n, u=None, tol=1e-8, max_steps=10 ** 7,
                       want_moments=False) -> int:
    nx, ny, nz = (int(v) for v in lattice)
    shape = (nz, ny, nx)
    nn = _f64(n, shape)
    uu = None if u is None else _f64(u, (3,) + shape)
    r = wdlb_request()
    r.desc = _desc(lattice, sigma, walls, tau, g)
    r.n = nn.ctypes.data
    r.u = None if uu is None else uu.ctypes.data
    r.tol = float(tol)
    r.max_steps = int(max_steps)
    outs = None
    if want_moments:
        outs = (np.zeros(shape), np.zeros((3,) + shape))
        r.out_n = outs[0].ctypes.data
        r.out_u = outs[1].ctypes.data
    rid = ctypes.c_int64()
    st = load_library().wdlb_server_submit(server.handle, ctypes.byref(r), ctypes.byref(rid))
    if st != WDLB_OK:
        raise WDLBError(st, "wdlb_server_submit")
    server.keep[rid.value] = outs
    server.nodes[rid.value] = nx * ny * nz
    return rid.value


def wdlb_server_poll(server, cap=1024, log=None):
    """Finished results: list of dicts (with 'n', 'u' if moments were
    requested).  log: a writable text file that receives one JSON line per
    finished solve (id, status, steps, residual, queue, run and total seconds,
    nodes, MLUPS of the solve, mean density, flux, effective viscosity)."""
    buf = (wdlb_result * cap)()
    k = load_library().wdlb_server_poll(server.handle, buf, cap)
    out = []
    for r in buf[:k]:
        d = {"id": r.id, "status": r.status, "steps": r.steps, "residual": r.residual, "submit_s": r.submit_s,
             "start_s": r.start_s, "finish_s": r.finish_s,
             "stats": {f: getattr(r.stats, f) for f, _ in wdlb_pore_stats._fields_}}
        outs = server.keep.pop(r.id, None)
        if outs is not None:
            d["n"], d["u"] = outs
        nodes = server.nodes.pop(r.id, 0)
        if log is not None:
            run_s = r.finish_s - r.start_s
            rec = {"id": r.id, "status": STATUS_NAMES.get(r.status, r.status), "steps": r.steps,
                   "residual": r.residual, "queue_s": r.start_s - r.submit_s, "run_s": run_s,
                   "latency_s": r.finish_s - r.submit_s, "nodes": nodes,
                   "mlups": nodes * r.steps / run_s / 1e6 if run_s > 0 else None,
                   "mean_n": r.stats.mean_n, "flux_x": r.stats.flux_x, "eta_eff": r.stats.eta_eff}
            log.write(json.dumps(rec) + "\n")
        out.append(d)
    if log is not None:
        log.flush()
    return out


def wdlb_server_info(server) -> dict:
    st = wdlb_server_stats()
    load_library().wdlb_server_info(server.handle, ctypes.byref(st))
    return {f: getattr(st, f) for f, _ in wdlb_server_stats._fields_}


def wdlb_server_destroy(server):
    if server.handle:
        load_library().wdlb_server_destroy(server.handle)
        server.handle = None


wdlb_result._fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("steps", ctypes.c_int64),
                        ("residual", ctypes.c_double), ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                        ("finish_s", ctypes.c_double), ("stats", wdlb_pore_stats)]
