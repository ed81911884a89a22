"""The benchmark's batched configuration at full size, in the launch
configuration bench.py times: the 64 slit pores of synth.batched_pores()
(32 x 32 x 13..121, sigma 4, n* in [0.1, 0.57]) in one FP32 batch on the
built-in tile rule (one shell launch for all pores, TMA tiles), stepped
through CUDA-graph replays.  Every pore's status must stay OK, and sampled
pores (the four smallest, which the oracle steps in seconds) must match the
FP64 oracle run on the same seeded inputs within the FP32 slit bounds of
test_gpu_parity (n 1e-6 relative; u 5e-4 of max|u|).  The same batch on the
persistent dataflow kernel gives bitwise the same populations."""
import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

pytestmark = pytest.mark.gpu

STEPS = 20


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def _batch(w, pores, persistent):
    b = w.wdlb_batch_create(len(pores), 2 << 30, storage="f32", autotune=False, persistent=persistent)
    slots = [w.wdlb_batch_add(b, (pp["nx"], pp["ny"], pp["nz"]), pp["sigma"], pp["walls"], pp["tau"], pp["g"], n, u)
             for pp, n, u in pores]
    return b, slots


def test_bench_batch_against_oracle(w, oracle_mod):
    pores = synth.batched_pores()
    b, slots = _batch(w, pores, False)
    assert all(w.wdlb_staging_info(w.wdlb_batch_context(b, s)) for s in slots)
    w.wdlb_batch_step(b, STEPS)
    _, st = w.wdlb_batch_residuals(b, 1)
    assert all(int(st[s]) == 0 for s in slots), st
    sizes = [pp["nx"] * pp["ny"] * pp["nz"] for pp, _, _ in pores]
    sample = sorted(range(len(pores)), key=lambda k: sizes[k])[:4]
    for k in sample:
        pp, n, u = pores[k]
        o = oracle_mod.Oracle(**pp)
        o.init(n, u)
        o.step(STEPS)
        n_o, u_o = o.moments()
        n_g, u_g = w.wdlb_moments(w.wdlb_batch_context(b, slots[k]))
        fl = slice(1, -1)
        en = np.max(np.abs(n_g[fl] - n_o[fl]) / n_o[fl])
        eu = np.max(np.abs(u_g[:, fl] - u_o[:, fl])) / np.abs(u_o[:, fl]).max()
        print("pore %d (nz %d, n* %.3f): n %.2e, u %.2e" % (k, pp["nz"], n_o[fl].mean() * 64, en, eu))
        assert en < 1e-6 and eu < 5e-4, (k, en, eu)
    f_graph = [w.wdlb_get_populations(w.wdlb_batch_context(b, s)) for s in slots[:8]]
    w.wdlb_batch_destroy(b)
    bp, pslots = _batch(w, pores, True)
    w.wdlb_batch_step(bp, STEPS)
    for s, f in zip(pslots[:8], f_graph):
        assert np.array_equal(w.wdlb_get_populations(w.wdlb_batch_context(bp, s)), f)
    w.wdlb_batch_destroy(bp)
