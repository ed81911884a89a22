"""The energy-equation fields on a prescribed temperature (wdlb_thermal_fields:
Q of Eq. campob1, B of Eq. campos, F^T of Eq. thermalforce) through the C ABI
against the FP64 oracle on the same seeded states: FP64 storage to 1e-11 and
FP32 storage to 1e-5 of each field's largest magnitude, in slits and periodic
boxes, with both shell rules, after a few steps (so the field velocity is the
predictor's).  A non-positive temperature on a fluid node is refused."""
import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


CASES = {
    "slit_s4": ((16, 12, 21), 4.0, True, "full"),
    "bulk_s3": ((14, 11, 13), 3.0, False, "full"),
    "slit_s4_compact": ((12, 12, 19), 4.0, True, "compact"),
}


def _state(lat, sigma, walls, seed):
    nx, ny, nz = lat
    n, _ = synth.uniform_with_noise(nx, ny, nz, 0.4 / sigma ** 3, 3e-2, seed, walls)
    rng = np.random.default_rng(seed)
    u = 1e-3 * rng.standard_normal((3, nz, ny, nx))
    T = (1.0 / 3.0) * (1 + 0.1 * rng.standard_normal((nz, ny, nx)))
    if walls:
        u[:, 0] = u[:, -1] = 0
    return n, u, T


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-5)])
@pytest.mark.parametrize("case", list(CASES))
def test_thermal_fields_match_oracle(w, oracle_mod, case, storage, tol):
    lat, sigma, walls, rule = CASES[case]
    n, u, T = _state(lat, sigma, walls, 17)
    g = (1e-5, 0.0, 0.0)
    ctx = w.wdlb_create(lat, sigma, walls, 0.9, g, storage=storage, shell_rule=rule)
    w.wdlb_init_fields(ctx, n, u)
    o = oracle_mod.Oracle(*lat, walls, sigma, 0.9, g, shell_rule=rule)
    o.init(n, u)
    w.wdlb_step(ctx, 3)
    o.step(3)
    got = w.wdlb_thermal_fields(ctx, T)
    want = o.thermal_fields(T)
    for name, a, b in zip(("Q", "B", "FT"), got, want):
        scale = np.abs(b).max()
        assert scale > 0, name
        err = np.abs(a - b).max() / scale
        print("%s %s %s: %.2e" % (case, storage, name, err))
        assert err < tol, (name, err)
    # B and F^T carry the same shell sum: B = 4 T n F^T on every fluid node
    n_g, _ = w.wdlb_moments(ctx)
    fl = slice(1, -1) if walls else slice(None)
    ratio = got[1][:, fl] / (4 * T[fl] * n_g[fl] * got[2][:, fl])
    bound = 1e-12 if storage == "f64" else 1e-6
    assert np.abs(ratio - 1).max() < bound
    w.wdlb_destroy(ctx)


def test_uniform_temperature_gives_no_heat_flux(w):
    lat = (16, 12, 21)
    n, u, _ = _state(lat, 4.0, True, 3)
    ctx = w.wdlb_create(lat, 4.0, True, 1.0, (0.0, 0.0, 0.0), storage="f32")
    w.wdlb_init_fields(ctx, n, u)
    _, B, FT = w.wdlb_thermal_fields(ctx, np.full(n.shape, 0.3))
    assert np.abs(B).max() == 0 and np.abs(FT).max() == 0
    w.wdlb_destroy(ctx)


def test_non_positive_temperature_is_refused(w):
    lat = (16, 12, 21)
    n, u, T = _state(lat, 4.0, True, 5)
    ctx = w.wdlb_create(lat, 4.0, True, 1.0, (0.0, 0.0, 0.0), storage="f32")
    w.wdlb_init_fields(ctx, n, u)
    T[5, 3, 2] = 0.0
    with pytest.raises(w.WDLBError) as ei:
        w.wdlb_thermal_fields(ctx, T)
    assert ei.value.status == 1
    T[5, 3, 2] = 0.3
    T[0] = -1.0                 # solid plane: ignored
    w.wdlb_thermal_fields(ctx, T)
    w.wdlb_destroy(ctx)


def test_collisional_conductivity_on_the_gpu(w, oracle_mod):
    """Q on a sinusoidal temperature in a uniform fluid at rest, through the
    CUDA path (FP64 storage), extrapolated to long waves: the collisional
    conductivity of Eq. thermalcond, (2/3) sqrt(pi T) g2 n^2 sigma^4, times the
    shell's second-moment ratio sum_e w e_x^2 / (4 pi sigma^2 / 3)."""
    sigma, nstar, T0, a = 4.0, 0.4, 0.35, 1e-4
    n0 = nstar / sigma ** 3
    chi = np.pi * sigma ** 3 / 6 * n0
    g2 = (1 - 0.5 * chi) / (1 - chi) ** 3
    e, wsh = oracle_mod.shell(sigma)
    ratio = float(np.sum(wsh * e[:, 0] ** 2)) / (4 * np.pi * sigma ** 2 / 3)
    vals = []
    for L in (128, 256):
        kappa = 2 * np.pi / L
        ctx = w.wdlb_create((L, 8, 8), sigma, False, 1.0, (0.0, 0.0, 0.0), storage="f64")
        w.wdlb_init_fields(ctx, np.full((8, 8, L), n0))
        T = np.broadcast_to(T0 + a * np.sin(kappa * np.arange(L)), (8, 8, L))
        Qf, _, _ = w.wdlb_thermal_fields(ctx, T)
        w.wdlb_destroy(ctx)
        vals.append(Qf[0, 0, L // 4] / (-a * kappa ** 2) / np.sqrt(T0 + a))
    got = (4 * vals[1] - vals[0]) / 3
    want = (2.0 / 3.0) * np.sqrt(np.pi) * g2 * n0 ** 2 * sigma ** 4 * ratio
    print("lambda_c / sqrt(T): GPU %.10e, paper x shell ratio %.10e (ratio %.4f)" % (got, want, ratio))
    assert abs(got / want - 1) < 2e-5
