"""The pore-viscosity sweep of Sec. 5 (Fig. 2's experiment) on the GPU.

The paper reports that the viscosity measured in a slit is consistently lower
than the bulk value in narrow slabs and converges to it for widths of the
order of 200 lattice units.  The sweep (steady Poiseuille flow through the
serving loop) must show that shape at packing fractions 0.11 and 0.32, and
its effective viscosity must equal the FP64 oracle's on the exact column for
two of the widths."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIGMA, TAU, GX = 4.0, 1.0, 1e-6


@pytest.fixture(scope="module")
def sweeps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, sweeps
    build.build()
    return sweeps


@pytest.mark.parametrize("chi", [0.11, 0.32])
def test_pore_viscosity_rises_to_the_bulk_value(sweeps, chi):
    widths = [8, 24, 64, 200]
    res = sweeps.pore_viscosity_sweep(chi, widths, sigma=SIGMA, tau=TAU, gx=GX)
    assert all(r["status"] == 0 for r in res), res
    ratio = np.array([r["ratio"] for r in res])
    print("chi %g: eta_eff / eta_bulk at H = %s: %s" % (chi, widths, np.round(ratio, 4)))
    assert np.all(np.diff(ratio) > 0)              # rises with the width
    assert ratio[-1] < 1.0 and ratio[-1] > 0.93    # near the bulk value at H = 200
    assert ratio[0] < 0.8 * ratio[-1]              # clearly lower in the narrowest slab


@pytest.mark.parametrize("chi,H", [(0.11, 16), (0.32, 24)])
def test_sweep_point_matches_oracle(sweeps, oracle_mod, chi, H):
    """A sweep width converged on both sides (the flux criterion can pass
    before a dense slit's density layering has relaxed, so the GPU lattice
    runs twice the oracle's step count): effective viscosity within the FP32
    slit bound, 2e-4.  Measured 2.3e-5 (chi 0.11, H 16) and 6.1e-5 (chi 0.32,
    H 24); 1.7e-4 and 1.0e-4 before the FP32 collision restored its in-plane
    momentum (in such thin slits the wall layers are a large part of the
    pore)."""
    from paper_1304_7880_gb300 import synth
    from paper_1304_7880_gb300 import wdlb as w
    nz = H + 2
    n0 = synth.packing_to_density(chi, SIGMA)
    n = np.full((nz, 1, 1), n0)
    n[0] = n[-1] = 0.0
    o = oracle_mod.Oracle(1, 1, nz, True, SIGMA, TAU, (GX, 0.0, 0.0))
    o.init(n)
    prev, steps = None, 0
    for _ in range(3000):
        o.step(100)
        steps += 100
        nn, uu = o.moments()
        q = float(np.sum(nn[1:-1] * uu[0, 1:-1]))
        if prev is not None and abs(q - prev) < 1e-13 * 100 * abs(q):
            break
        prev = q
    ref = oracle_mod.pore_average(nn, uu, True, GX)
    ctx = w.wdlb_create((8, 8, nz), SIGMA, True, TAU, (GX, 0.0, 0.0), storage="f32")
    w.wdlb_init_fields(ctx, np.broadcast_to(n, (nz, 8, 8)).copy())
    w.wdlb_step(ctx, 2 * steps)
    st = w.wdlb_pore_average(ctx)
    w.wdlb_destroy(ctx)
    print("chi %.2f H %d: eta_eff rel err %.2e" % (chi, H, st["eta_eff"] / ref["eta_eff"] - 1))
    assert st["eta_eff"] == pytest.approx(ref["eta_eff"], rel=2e-4)
    assert st["mean_n"] == pytest.approx(ref["mean_n"], rel=1e-6)
    assert st["eta_eff"] / sweeps.bulk_shear_viscosity(st["mean_n"], SIGMA, TAU) < 1.0


def test_bulk_viscosity_sweep_matches_theory_and_the_cross_over_raises_it(sweeps):
    """The bulk shear viscosity at sigma = 8 (Sec. 5, Fig. 1's experiment):
    measured from the decay of a transverse wave, it follows the long-wave
    closed form (1 %), grows with the packing fraction, and the cross-over
    term (K = 2) makes it larger than without it (K = 0) at every density, as
    the paper reports."""
    res = sweeps.bulk_viscosity_sweep([0.1, 0.25, 0.35])
    for r in res:
        assert r["eta"] == pytest.approx(r["eta_theory"], rel=1e-2), r
    eta = {(r["chi"], r["K"]): r["eta"] for r in res}
    for chi in (0.1, 0.25, 0.35):
        assert eta[(chi, 2.0)] > eta[(chi, 0.0)]
    assert eta[(0.1, 2.0)] < eta[(0.25, 2.0)] < eta[(0.35, 2.0)]


def test_bulk_viscosity_point_matches_oracle(sweeps, oracle_mod):
    """chi = 0.25, K = 2, sigma = 8: the same decay measurement on the
    oracle's exact 1 x 1 x 256 column gives the same viscosity (1e-3)."""
    import math
    from paper_1304_7880_gb300 import synth
    chi, K, L, sigma, tau = 0.25, 2.0, 256, 8.0, 1.0
    gpu = sweeps.bulk_viscosity_sweep([chi], k_values=(K,))[0]
    n0 = synth.packing_to_density(chi, sigma)
    q = 2 * math.pi / L
    sz = np.sin(q * np.arange(L))
    rate_th = sweeps.bulk_shear_viscosity(n0, sigma, tau, K) / n0 * q * q
    span = int(math.ceil(1.0 / rate_th))
    every = max(1, span // 8)
    o = oracle_mod.Oracle(1, 1, L, False, sigma, tau, k_cross=K)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = 1e-6 * sz
    o.init(np.full((L, 1, 1), n0), u)
    o.step(span // 10)
    t, a = [], []
    for k in range(9):
        if k:
            o.step(every)
        t.append(span // 10 + k * every)
        a.append(2.0 / L * float(np.sum(o.moments()[1][0, :, 0, 0] * sz)))
    eta_oracle = n0 * (-np.polyfit(t, np.log(a), 1)[0]) / (q * q)
    assert gpu["eta"] == pytest.approx(eta_oracle, rel=1e-3)


def test_compact_shell_pore_viscosity_against_the_full_shell(sweeps):
    """The compact contact shell in confinement (chi = 0.11, sigma 4): it lowers
    the effective viscosity of a narrow slit (the wall layers are
    finite-wavenumber structure, where the two quadratures differ) and meets the
    full shell's value in a wide one (both tend to their common long-wave bulk
    viscosity)."""
    full = sweeps.pore_viscosity_sweep(0.11, [8, 200])
    comp = sweeps.pore_viscosity_sweep(0.11, [8, 200], shell_rule="compact")
    assert all(r["status"] == 0 for r in full + comp)
    assert comp[0]["ratio"] < full[0]["ratio"] < comp[1]["ratio"]
    assert comp[1]["ratio"] == pytest.approx(full[1]["ratio"], rel=0.01)
    assert comp[1]["ratio"] > 0.95
