"""GPU parity of the compact contact shell (two or three cubic orbits with
per-orbit weights; the quadrature of the integral over khat in Eq. campoc that
keeps the virial coefficient, the long-wave shear viscosity and a fourth-rank
isotropic moment) against the FP64 oracle running the same rule.

Tolerances are those of the full shell (test_gpu_parity): FP64 1e-10, FP32
1e-5 on n and u in bulk boxes, FP16 n 1e-6 / u 5e-3 (bulk; FP16 is refused
in slits).  Batches with the compact rule step bit-identically alone and
batched.
"""
import math

import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-10, 1e-10), "f32": (1e-5, 1e-5), "f16": (1e-6, 5e-3)}


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def make_pair(w, oracle_mod, p, n, u, storage, **opt):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ctx = w.wdlb_create((nx, ny, nz), p["sigma"], p["walls"], p["tau"], p["g"], storage=storage,
                        shell_rule="compact", **opt)
    w.wdlb_init_fields(ctx, n, u)
    o = oracle_mod.Oracle(nx, ny, nz, p["walls"], p["sigma"], p["tau"], p["g"], shell_rule="compact")
    o.init(n, u)
    return ctx, o


def fluid(shape, walls):
    m = np.ones(shape, dtype=bool)
    if walls:
        m[0] = m[-1] = False
    return m


def compare(ctx, o, walls, tol, w):
    n_g, u_g = w.wdlb_moments(ctx)
    n_o, u_o = o.moments()
    m = fluid(n_o.shape, walls)
    en = np.max(np.abs(n_g[m] - n_o[m]) / np.abs(n_o[m]))
    eu = np.max(np.abs(u_g[:, m] - u_o[:, m])) / np.abs(u_o[:, m]).max()
    assert en <= tol[0], "n: %.3e > %.1e" % (en, tol[0])
    assert eu <= tol[1], "u: %.3e > %.1e" % (eu, tol[1])
    return en, eu


def noisy_state(p, nstar, amp, seed):
    n, _ = synth.uniform_with_noise(p["nx"], p["ny"], p["nz"], nstar / p["sigma"] ** 3, amp, seed, p["walls"])
    rng = np.random.default_rng(seed)
    u = 1e-3 * rng.standard_normal((3,) + n.shape)
    if p["walls"]:
        u[:, 0] = u[:, -1] = 0
    return n, u


@pytest.mark.parametrize("case", ["bulk_s3", "slit_s4", "bulk_s8"])
def test_compact_fields_match_oracle_f64(w, oracle_mod, case):
    p = {"bulk_s3": dict(nx=9, ny=8, nz=7, walls=False, sigma=3.0, tau=0.9, g=(1e-5, 0, 0)),
         "slit_s4": dict(nx=8, ny=8, nz=21, walls=True, sigma=4.0, tau=1.0, g=(1e-5, 0, 0)),
         "bulk_s8": dict(nx=10, ny=9, nz=17, walls=False, sigma=8.0, tau=1.0, g=(0, 1e-5, 0))}[case]
    n, u = noisy_state(p, 0.5, 5e-2, 3)
    ctx, o = make_pair(w, oracle_mod, p, n, u, "f64")
    for _ in range(2):
        nb_g, C_g, A_g, _ = w.wdlb_fields(ctx)
        nb_o, C_o, A_o = o.fields()
        m = fluid(nb_o.shape, p["walls"])
        np.testing.assert_allclose(nb_g[m], nb_o[m], rtol=1e-12)
        np.testing.assert_allclose(C_g[:, m], C_o[:, m], rtol=0, atol=1e-11 * np.abs(C_o).max())
        np.testing.assert_allclose(A_g[:, m], A_o[:, m], rtol=0, atol=1e-11 * np.abs(A_o).max())
        w.wdlb_step(ctx, 3)
        o.step(3)


TILED = {
    "s3_periodic_13x11x19": dict(nx=13, ny=11, nz=19, walls=False, sigma=3.0, tau=0.8, g=(0, 1e-5, 0)),
    "s4_periodic_17x9x12": dict(nx=17, ny=9, nz=12, walls=False, sigma=4.0, tau=1.0, g=(0, 0, 1e-5)),
    "s4_slit_10x8x27": dict(nx=10, ny=8, nz=27, walls=True, sigma=4.0, tau=1.0, g=(1e-5, 0, 0)),
    "s6_slit_12x9x35": dict(nx=12, ny=9, nz=35, walls=True, sigma=6.0, tau=1.0, g=(1e-5, 0, 0)),
}


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("name", sorted(TILED))
def test_compact_tiled_fp32_ragged(w, oracle_mod, name, tile):
    """The tiled FP32 kernel with per-pair weights, every tile shape, ragged
    lattices (partial bricks, halos wrapping more than once, walls)."""
    p = TILED[name]
    n, u = noisy_state(p, 0.4, 2e-2, 17)
    ctx, o = make_pair(w, oracle_mod, p, n, u, "f32", tile=tile)
    assert w.wdlb_tile_info(ctx) == (True, tile)
    w.wdlb_step(ctx, 20)
    o.step(20)
    compare(ctx, o, p["walls"], TOL["f32"], w)


@pytest.mark.parametrize("name", sorted(TILED))
def test_compact_tiled_fp16_ragged(w, oracle_mod, name):
    p = TILED[name]
    if p["walls"]:
        pytest.skip("FP16 storage is for periodic boxes only")
    n, u = noisy_state(p, 0.4, 2e-2, 17)
    ctx, o = make_pair(w, oracle_mod, p, n, u, "f16")
    w.wdlb_step(ctx, 20)
    o.step(20)
    compare(ctx, o, p["walls"], TOL["f16"], w)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_compact_generic_kernel_sigma8(w, oracle_mod, storage):
    """sigma 8 (no tiled kernel: its halo does not fit in shared memory) runs
    the generic kernel with per-vector weights; 42 vectors instead of 762."""
    p = dict(nx=16, ny=16, nz=20, walls=False, sigma=8.0, tau=1.0, g=(1e-5, 0, 0))
    n, u = noisy_state(p, 0.4, 2e-2, 19)
    ctx, o = make_pair(w, oracle_mod, p, n, u, storage)
    assert w.wdlb_tile_info(ctx)[0] is False
    w.wdlb_step(ctx, 10)
    o.step(10)
    compare(ctx, o, False, TOL[storage], w)


def test_compact_slit_8x8x41_f64(w, oracle_mod):
    p, n, u = synth.slit_8x8x41()
    ctx, o = make_pair(w, oracle_mod, p, n, u, "f64")
    for _ in range(2):
        w.wdlb_step(ctx, 100)
        o.step(100)
        compare(ctx, o, True, TOL["f64"], w)


def test_compact_bulk_128_full_size(w, oracle_mod):
    """The 128^3 bulk workload with the compact shell (FP32, the launch
    configuration the benchmark times): two steps against the oracle on every
    node."""
    p, n, u = synth.bulk_shear_128()
    ctx, o = make_pair(w, oracle_mod, p, n, u, "f32")
    w.wdlb_step(ctx, 2)
    o.step(2)
    compare(ctx, o, False, TOL["f32"], w)


PORES = [
    ((16, 16, 25), 4.0, True, 1.0, (1e-5, 0, 0), 0.4, 31),
    ((12, 10, 19), 3.0, True, 0.8, (3e-6, 0, 0), 0.3, 33),
    ((16, 16, 40), 6.0, True, 1.0, (1e-6, 0, 0), 0.35, 36),
    ((6, 5, 21), 4.0, True, 1.0, (2e-6, 0, 0), 0.45, 35),
    ((16, 16, 20), 8.0, False, 1.0, (0, 0, 0), 0.3, 37),
]


def test_compact_batch_equals_alone(w):
    def fields(pore):
        lat, sigma, walls, tau, g, nstar, seed = pore
        return synth.uniform_with_noise(*lat, nstar / sigma ** 3, 1e-3, seed, walls)

    ref = []
    for pore in PORES:
        lat, sigma, walls, tau, g, _, _ = pore
        n, u = fields(pore)
        ctx = w.wdlb_create(lat, sigma, walls, tau, g, storage="f32", shell_rule="compact")
        w.wdlb_init_fields(ctx, n, u)
        w.wdlb_step(ctx, 7)
        ref.append(w.wdlb_get_populations(ctx))
        w.wdlb_destroy(ctx)
    b = w.wdlb_batch_create(8, 256 << 20, storage="f32", shell_rule="compact")
    slots = []
    for pore in PORES:
        lat, sigma, walls, tau, g, _, _ = pore
        n, u = fields(pore)
        slots.append(w.wdlb_batch_add(b, lat, sigma, walls, tau, g, n, u))
    w.wdlb_batch_step(b, 7)
    for s, f_ref in zip(slots, ref):
        f = w.wdlb_get_populations(w.wdlb_batch_context(b, s))
        assert np.array_equal(f, f_ref)
    w.wdlb_batch_destroy(b)


def test_checkpoint_refuses_another_shell_rule(w):
    p, n, u = synth.slit_8x8x41()
    a = w.wdlb_create((8, 8, 41), 4.0, True, p["tau"], p["g"], shell_rule="compact")
    w.wdlb_init_fields(a, n, u)
    w.wdlb_step(a, 5)
    blob = w.wdlb_save_state(a)
    b = w.wdlb_create((8, 8, 41), 4.0, True, p["tau"], p["g"], shell_rule="full")
    w.wdlb_init_fields(b, n, u)
    with pytest.raises(w.WDLBError):
        w.wdlb_load_state(b, blob)
    c = w.wdlb_create((8, 8, 41), 4.0, True, p["tau"], p["g"], shell_rule="compact")
    w.wdlb_init_fields(c, n, u)
    w.wdlb_load_state(c, blob)
    w.wdlb_step(a, 3)
    w.wdlb_step(c, 3)
    assert np.array_equal(w.wdlb_get_populations(a), w.wdlb_get_populations(c))


def test_compact_bulk_viscosity_sweep_is_the_continuum_value(w):
    """sigma 8, the transverse-wave decay of the bulk sweep: with the compact
    shell the long-wave viscosity is the continuum closed form of Sec. 4,
    eta = n [kT (tau-1/2) + (tau-1/2) K kT n g2 4 pi sigma^3/15
             + beta g2 n 2 pi sigma^2/15]."""
    from paper_1304_7880_gb300 import sweeps
    kT, sigma, tau = 1.0 / 3.0, 8.0, 1.0
    beta = 2 * sigma ** 2 * math.sqrt(kT / math.pi)
    res = sweeps.bulk_viscosity_sweep([0.1, 0.25], sigma=sigma, shell_rule="compact")
    for r in res:
        n, K = r["n"], r["K"]
        g2 = sweeps.contact_value(r["chi"])
        cont = n * (kT * (tau - 0.5) + (tau - 0.5) * K * kT * n * g2 * 4 * math.pi * sigma ** 3 / 15
                    + beta * g2 * n * 2 * math.pi * sigma ** 2 / 15)
        assert r["eta_theory"] == pytest.approx(cont, rel=1e-12)
        assert r["eta"] == pytest.approx(cont, rel=5e-3)


@pytest.mark.parametrize("case", ["s3.5_f64", "s3.5_f32", "s2_f64", "py_closure_f64"])
def test_compact_generic_kernel_edge_cases(w, oracle_mod, case):
    """The generic shell kernel with per-vector weights where the tiled kernel
    does not apply: sigma 3.5 (no compiled tile), sigma 2 (the smallest sigma
    with a compact rule, 38 vectors), the Percus-Yevick closure."""
    sigma = {"s3.5_f64": 3.5, "s3.5_f32": 3.5, "s2_f64": 2.0, "py_closure_f64": 4.0}[case]
    storage = "f32" if case.endswith("f32") else "f64"
    closure = "PY" if case.startswith("py") else "CS"
    p = dict(nx=11, ny=9, nz=15, walls=True, sigma=sigma, tau=0.9, g=(1e-5, 0, 0))
    n, u = noisy_state(p, 0.4, 2e-2, 29)
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ctx = w.wdlb_create((nx, ny, nz), sigma, True, p["tau"], p["g"], storage=storage, closure=closure,
                        shell_rule="compact")
    w.wdlb_init_fields(ctx, n, u)
    assert w.wdlb_tile_info(ctx)[0] is False
    o = oracle_mod.Oracle(nx, ny, nz, True, sigma, p["tau"], p["g"], closure=closure, shell_rule="compact")
    o.init(n, u)
    w.wdlb_step(ctx, 15)
    o.step(15)
    compare(ctx, o, True, TOL[storage], w)
