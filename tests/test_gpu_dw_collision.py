"""The double-word collision (wdlb_options.collision = WDLB_COLLISION_DW): FP32
population storage with the collision and the push's re-encoding in pairs of
floats, rounded to FP32 once at the store.

* Against the FP64 oracle: the converged 256 x 256 x 161 slit (8 x 8
  cross-section, three times the oracle's steps) at n* 0.3 and 0.6 within
  1e-5 on n, u_x and the pore flux (the FP32 collision without its in-plane
  momentum correction: up to 5.4e-5); a
  short run of a noisy slit and the plain slit of Sec. 5's experiment at
  8 x 8 x 41 after 1000 steps within the FP32 slit bounds (there the 3-D
  flows the noise drives carry the FP32 fields' rounding, as with the FP32
  collision: u_x ~1e-4 of max|u_x| pointwise; the flux within 1e-5).  u is
  relative to max|u_x|.
* A batch of double-word pores steps every pore bit for bit as it steps alone,
  and the persistent dataflow kernel as the per-phase launches.
* The library refuses the option for periodic boxes and for FP16 and FP64
  storage (WDLB_ERR_ARG).
"""
import os

import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

from oracle_views import collision_velocity

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "slit_column_steady.txt")


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def _pair(w, oracle_mod, p, n, u, **opt):
    lat = (p["nx"], p["ny"], p["nz"])
    ctx = w.wdlb_create(lat, p["sigma"], p["walls"], p["tau"], p["g"], storage="f32", collision="dw", **opt)
    w.wdlb_init_fields(ctx, n, u)
    o = oracle_mod.Oracle(p["nx"], p["ny"], p["nz"], p["walls"], p["sigma"], p["tau"], p["g"])
    o.init(n, u)
    return ctx, o


def _errors(w, ctx, o):
    n_g, u_g = w.wdlb_moments(ctx)
    n_o, u_o = o.moments()
    fl = slice(1, -1)
    umax = np.abs(u_o[0, fl]).max()
    en = np.max(np.abs(n_g[fl] - n_o[fl]) / n_o[fl])
    ec = [np.abs(u_g[a, fl] - u_o[a, fl]).max() / umax for a in range(3)]
    return en, ec


def test_dw_short_run_against_oracle(w, oracle_mod):
    """A sigma-4 slit with 2 % density noise and random velocities, 20 steps."""
    lat = (16, 16, 25)
    n, u = synth.uniform_with_noise(*lat, 0.45 / 64, 2e-2, 5, True)
    rng = np.random.default_rng(5)
    u = 1e-3 * rng.standard_normal(u.shape)
    u[:, 0] = u[:, -1] = 0
    p = dict(nx=16, ny=16, nz=25, sigma=4.0, walls=True, tau=0.9, g=(1e-5, 0.0, 0.0))
    ctx, o = _pair(w, oracle_mod, p, n, u)
    w.wdlb_step(ctx, 20)
    o.step(20)
    en, ec = _errors(w, ctx, o)
    print("dw 16x16x25 20 steps: n %.2e, u_x %.2e, u_y %.2e, u_z %.2e" % (en, *ec))
    assert en < 1e-6 and max(ec) < 5e-4          # measured u_z 2.1e-4, as with the FP32 collision
    w.wdlb_destroy(ctx)


def test_dw_slit_8x8x41(w, oracle_mod):
    p, n, u = synth.slit_8x8x41()
    ctx, o = _pair(w, oracle_mod, p, n, u)
    for _ in range(10):
        w.wdlb_step(ctx, 100)
        o.step(100)
    en, ec = _errors(w, ctx, o)
    st = w.wdlb_pore_average(ctx)
    n_o, u_o = o.moments()
    ref = oracle_mod.pore_average(n_o, u_o, True, p["g"][0])
    ef = abs(st["flux_x"] - ref["flux_x"]) / abs(ref["flux_x"])
    uc_g = w.wdlb_fields(ctx)[3]
    uc_o = collision_velocity(oracle_mod, o, p["g"])
    fl = slice(1, -1)
    ecc = [np.abs(uc_g[a, fl] - uc_o[a, fl]).max() / np.abs(uc_o[0, fl]).max() for a in range(3)]
    print("dw 8x8x41 1000 steps: n %.2e, u_x %.2e, u_y %.2e, u_z %.2e, flux %.2e; collision u_x %.2e, u_y %.2e, "
          "u_z %.2e" % (en, *ec, ef, *ecc))
    assert en < 1e-6 and ef < 1e-5 and max(ec) < 5e-4    # measured flux 3.1e-6, u_x 1.0e-4, u_z 4.2e-4
    assert max(ecc) < 5e-4                               # measured u_x 1.0e-4, u_z 2.5e-4
    w.wdlb_destroy(ctx)


def _golden():
    out, cur = {}, None
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split(":", 1)
            if key == "n_star":
                cur = float(val)
                out[cur] = {}
            elif key == "steps":
                out[cur]["steps"] = int(val)
            else:
                out[cur][key] = np.array([float(v) for v in val.split()])
    return out


@pytest.mark.parametrize("n_star", [0.3, 0.6])
def test_dw_steady_slit_256x256x161(w, n_star):
    """The converged slit configuration (sigma 4, tau 0.8, g_x 1e-6) from a
    uniform start, on an 8 x 8 cross-section (the state stays uniform in x
    and y), three times the oracle's steps."""
    ref = _golden()[n_star]
    nz = 161
    n = np.full((nz, 8, 8), n_star / 64)
    n[0] = n[-1] = 0.0
    ctx = w.wdlb_create((8, 8, nz), 4.0, True, 0.8, (1e-6, 0.0, 0.0), storage="f32", collision="dw")
    w.wdlb_init_fields(ctx, n)
    steps = 3 * ref["steps"]
    w.wdlb_step(ctx, steps)
    n_g, u_g = w.wdlb_moments(ctx)
    uc_g = w.wdlb_fields(ctx)[3]
    w.wdlb_destroy(ctx)
    n_z, u_z = n_g[1:-1, 0, 0], u_g[0, 1:-1, 0, 0]
    n_o, u_o = ref["n"][1:-1], ref["ux"][1:-1]
    en = np.max(np.abs(n_z - n_o) / n_o)
    eu = np.max(np.abs(u_z - u_o)) / np.abs(u_o).max()
    eq = abs(np.sum(n_z * u_z) / np.sum(n_o * u_o) - 1)
    # converged: the collision velocity u equals the oracle's v (reading R7)
    euc = np.max(np.abs(uc_g[0, 1:-1, 0, 0] - u_o)) / np.abs(u_o).max()
    print("dw n* %g: %d steps, n %.2e, u_x %.2e, flux %.2e, collision u_x %.2e" % (n_star, steps, en, eu, eq, euc))
    assert en < 1e-6 and eu < 1e-5 and eq < 1e-5 and euc < 1e-5


PORES = [((16, 16, 25), 1e-5, 0.4, 41), ((32, 24, 61), 3e-6, 0.5, 42), ((8, 8, 41), 1e-6, 0.3, 43),
         ((24, 16, 17), 2e-6, 0.45, 44)]


def _pore(k):
    lat, g, nstar, seed = PORES[k]
    n, u = synth.uniform_with_noise(*lat, nstar / 64, 1e-3, seed, True)
    return lat, (g, 0.0, 0.0), n, u


@pytest.mark.parametrize("persistent", [False, True])
def test_dw_batch_equals_alone(w, persistent):
    alone = []
    for k in range(len(PORES)):
        lat, g, n, u = _pore(k)
        ctx = w.wdlb_create(lat, 4.0, True, 1.0, g, storage="f32", collision="dw", autotune=False)
        w.wdlb_init_fields(ctx, n, u)
        w.wdlb_step(ctx, 37)
        alone.append(w.wdlb_get_populations(ctx))
        w.wdlb_destroy(ctx)
    b = w.wdlb_batch_create(8, 256 << 20, storage="f32", autotune=False, persistent=persistent, collision="dw")
    slots = []
    for k in range(len(PORES)):
        lat, g, n, u = _pore(k)
        slots.append(w.wdlb_batch_add(b, lat, 4.0, True, 1.0, g, n, u))
    w.wdlb_batch_step(b, 37)
    _, st = w.wdlb_batch_residuals(b, 1)
    assert all(int(st[s]) == 0 for s in slots), st
    for k, s in enumerate(slots):
        assert np.array_equal(w.wdlb_get_populations(w.wdlb_batch_context(b, s)), alone[k]), k
    w.wdlb_batch_destroy(b)


def test_dw_refused_outside_fp32_slits(w):
    for walls, storage in ((False, "f32"), (True, "f64"), (False, "f16")):
        with pytest.raises(w.WDLBError) as ei:
            w.wdlb_create((16, 16, 16), 4.0, walls, 1.0, (0.0, 0.0, 0.0), storage=storage, collision="dw")
        assert ei.value.status == 1
    for storage in ("f64", "f16"):
        with pytest.raises(w.WDLBError) as ei:
            w.wdlb_batch_create(2, 64 << 20, storage=storage, collision="dw")
        assert ei.value.status == 1
    b = w.wdlb_batch_create(2, 64 << 20, storage="f32", collision="dw")
    n, u = synth.uniform_with_noise(16, 16, 16, 0.3 / 64, 1e-3, 1, False)
    with pytest.raises(w.WDLBError) as ei:
        w.wdlb_batch_add(b, (16, 16, 16), 4.0, False, 1.0, (0.0, 0.0, 0.0), n, u)
    assert ei.value.status == 1
    w.wdlb_batch_destroy(b)


@pytest.mark.parametrize("closure,omega_mode,collision", [("PY", "const", "dw"), ("CS", "nbar", "dw"),
                                                            ("CS", "nbar", "fp32")])
def test_dw_other_closures_and_relaxation_modes(w, oracle_mod, closure, omega_mode, collision):
    """The double-word collision on the generic shell kernel (Percus-Yevick
    closure) and with the relaxation rate from the smeared density (the FP32
    collision too), the reference density left to its default (the initial
    fluid mean): a noisy slit, 20 steps, against the oracle within the FP32
    slit bounds."""
    lat, g = (12, 10, 23), (1e-5, 0.0, 0.0)
    n, u = synth.uniform_with_noise(*lat, 0.4 / 64, 2e-2, 9, True)
    ctx = w.wdlb_create(lat, 4.0, True, 0.9, g, storage="f32", collision=collision, closure=closure,
                        omega_mode=omega_mode)
    w.wdlb_init_fields(ctx, n, u)
    o = oracle_mod.Oracle(*lat, True, 4.0, 0.9, g, closure=closure, omega_mode=omega_mode)
    o.init(n, u)
    w.wdlb_step(ctx, 20)
    o.step(20)
    en, ec = _errors(w, ctx, o)
    print("%s %s %s 20 steps: n %.2e, u_x %.2e, u_y %.2e, u_z %.2e" % (collision, closure, omega_mode, en, *ec))
    assert en < 1e-6 and max(ec) < 5e-4
    w.wdlb_destroy(ctx)
