"""The persistent dataflow step of a batch (one kernel per wdlb_batch_step
call; each pore's phases follow one another without device-wide barriers)
against the default step (one launch per phase, replayed from CUDA graphs).

Both run the same per-block bodies on the same work items, so the populations
must agree bit for bit: on uneven sigma-4 slits and a bulk box, through an odd
step count (buffer parity), an admission and a removal, and with the compact
shell.  A batch the persistent kernel does not serve (a sigma-3 pore) falls
back to the default step.  A dependency wait that cannot be met gives up
after its bound and every slot reports WDLB_ERR_TIMEOUT."""
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


# (lattice, walls, g, n*, seed), all sigma 4 (tau 1)
PORES = [
    ((16, 16, 25), True, (1e-5, 0, 0), 0.4, 41),
    ((32, 24, 61), True, (3e-6, 0, 0), 0.5, 42),
    ((8, 8, 41), True, (1e-6, 0, 0), 0.3, 43),
    ((24, 16, 17), True, (2e-6, 0, 0), 0.45, 44),
    ((40, 8, 33), True, (5e-6, 0, 0), 0.35, 45),
    ((16, 16, 20), False, (0, 0, 0), 0.5, 46),
]


def _add(w, b, k):
    lat, walls, g, nstar, seed = PORES[k]
    n, u = synth.uniform_with_noise(*lat, nstar / 64, 1e-3, seed, walls)
    return w.wdlb_batch_add(b, lat, 4.0, walls, 1.0, g, n, u)


def _run(w, persistent, keys, rule="full"):
    b = w.wdlb_batch_create(8, 256 << 20, storage="f32", autotune=False, persistent=persistent, shell_rule=rule)
    slots = {k: _add(w, b, k) for k in keys[:-1]}
    w.wdlb_batch_step(b, 37)
    w.wdlb_batch_remove(b, slots.pop(keys[0]))
    slots[keys[-1]] = _add(w, b, keys[-1])
    w.wdlb_batch_step(b, 24)
    _, st = w.wdlb_batch_residuals(b, 1)
    out = {k: w.wdlb_get_populations(w.wdlb_batch_context(b, s)) for k, s in slots.items()}
    assert all(int(st[s]) == 0 for s in slots.values()), st
    w.wdlb_batch_destroy(b)
    return out


@pytest.mark.parametrize("rule,keys", [("full", [0, 1, 2, 3, 4]), ("full", [5, 0, 1, 2]),
                                       ("compact", [0, 1, 3, 4])])
def test_persistent_step_equals_phase_launches(w, rule, keys):
    a = _run(w, False, keys, rule)
    b = _run(w, True, keys, rule)
    assert sorted(a) == sorted(b)
    for k in a:
        assert np.array_equal(a[k], b[k]), "pore %d" % k


def test_persistent_falls_back_for_other_kernels(w):
    """A sigma-3 pore makes a second shell group: the batch takes the per-phase
    launches and still steps every pore as the default batch does."""
    res = []
    for persistent in (False, True):
        b = w.wdlb_batch_create(4, 128 << 20, storage="f32", autotune=False, persistent=persistent)
        s0 = _add(w, b, 0)
        n, u = synth.uniform_with_noise(12, 10, 19, 0.3 / 27, 1e-3, 47, True)
        s1 = w.wdlb_batch_add(b, (12, 10, 19), 3.0, True, 0.8, (3e-6, 0, 0), n, u)
        w.wdlb_batch_step(b, 11)
        res.append([w.wdlb_get_populations(w.wdlb_batch_context(b, s)) for s in (s0, s1)])
        w.wdlb_batch_destroy(b)
    for x, y in zip(*res):
        assert np.array_equal(x, y)


def test_persistent_wait_that_runs_out_is_reported(w):
    """Every dependency wait asks for one item more than exists (tests only):
    each gives up after 16 tries, the kernel stops, and every slot reports the
    timeout instead of hanging."""
    b = w.wdlb_batch_create(4, 128 << 20, storage="f32", autotune=False, persistent=True, wait_limit=-16)
    slots = [_add(w, b, k) for k in (0, 2)]
    w.wdlb_batch_step(b, 3)
    _, st = w.wdlb_batch_residuals(b, 1)
    assert all(int(st[s]) == 5 for s in slots), st
    w.wdlb_batch_destroy(b)
