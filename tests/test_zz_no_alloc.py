"""wdlb_fields_static, the entry point that allocates no device memory (for
callers running inside another framework's memory pool or a host that forbids
cudaMalloc), against the FP64 oracle and against the allocating entry point
wdlb_fields on the same states.

A fresh state (populations at the local equilibrium of n and u, g = 0, no
history) has field velocity u, so the oracle's fields() and wdlb_fields of a
freshly initialised FP32 context both evaluate the fields that
wdlb_fields_static evaluates from device arrays n and u.  The static call runs
FP32 arithmetic; the bound is the FP32 tolerance of the parity tests, 1e-5 of
the largest magnitude.  Two calls in a row, on two different states, check that
the shared scratch array carries nothing from one call to the next.  The
cases span sigma 1 to 8 (8: 762 shell and 257 ball vectors, nearest the
array's table limits) and the three closures."""
import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def _state(shape, sigma, walls, seed):
    nz, ny, nx = shape
    n, u = synth.uniform_with_noise(nx, ny, nz, 0.5 / sigma ** 3, 5e-2, seed, walls)
    rng = np.random.default_rng(seed)
    u = 1e-3 * rng.standard_normal(u.shape)
    if walls:
        u[:, 0] = u[:, -1] = 0.0
    return n, u


def _static(w, shape, sigma, walls, closure, n, u):
    import torch
    nz, ny, nx = shape
    out_nb = torch.empty(shape, dtype=torch.float64, device="cuda")
    out_C = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    out_A = torch.empty((6,) + shape, dtype=torch.float64, device="cuda")
    d_n = torch.from_numpy(n).cuda()
    d_u = torch.from_numpy(u).cuda()
    torch.cuda.synchronize()
    w.wdlb_fields_static((nx, ny, nz), sigma, walls, closure, d_n, d_u, out_nb, out_C, out_A)
    torch.cuda.synchronize()
    return out_nb.cpu().numpy(), out_C.cpu().numpy(), out_A.cpu().numpy()


def _close(got, ref, mask):
    nb, C, A = got
    nb_ref, C_ref, A_ref = ref
    np.testing.assert_allclose(nb[mask], nb_ref[mask], rtol=TOL)
    np.testing.assert_allclose(C[:, mask], C_ref[:, mask], rtol=0, atol=TOL * np.abs(C_ref[:, mask]).max())
    np.testing.assert_allclose(A[:, mask], A_ref[:, mask], rtol=0, atol=TOL * np.abs(A_ref[:, mask]).max())
    if not mask.all():
        assert not C[:, ~mask].any() and not A[:, ~mask].any()


CASES = [
    # walls, (nz, ny, nx), sigma, closure
    (False, (24, 20, 16), 4.0, "CS"),
    (True, (33, 16, 16), 4.0, "CS"),
    (True, (21, 12, 10), 3.5, "PY"),
    (False, (9, 7, 8), 1.0, "ONE"),
    (True, (20, 16, 16), 8.0, "PY"),
    (False, (16, 16, 18), 8.0, "CS"),
]


@pytest.mark.parametrize("walls,shape,sigma,closure", CASES)
def test_fields_static_matches_oracle_and_fields(w, oracle_mod, walls, shape, sigma, closure):
    nz, ny, nx = shape
    mask = np.ones(shape, dtype=bool)
    if walls:
        mask[0] = mask[-1] = False
    for seed in (11, 12):                   # two calls in a row on different states
        n, u = _state(shape, sigma, walls, seed)
        got = _static(w, shape, sigma, walls, closure, n, u)
        o = oracle_mod.Oracle(nx, ny, nz, walls, sigma, 1.0, closure=closure)
        o.init(n, u)
        _close(got, o.fields(), mask)
        ctx = w.wdlb_create((nx, ny, nz), sigma, walls, 1.0, (0.0, 0.0, 0.0), storage="f32", closure=closure)
        w.wdlb_init_fields(ctx, n, u)
        nb_ref, C_ref, A_ref, _ = w.wdlb_fields(ctx)
        w.wdlb_destroy(ctx)
        _close(got, (nb_ref, C_ref, A_ref), mask)


def test_fields_static_reports_a_non_physical_state(w):
    """A uniform density whose packing fraction is above one (n* = 2.5) is
    reported as WDLB_ERR_UNSTABLE; the next valid call succeeds again."""
    shape, sigma = (10, 8, 8), 4.0
    n = np.full(shape, 2.5 / sigma ** 3)
    u = np.zeros((3,) + shape)
    with pytest.raises(w.WDLBError) as ei:
        _static(w, shape, sigma, False, "CS", n, u)
    assert ei.value.status == 4
    n, u = _state(shape, sigma, False, 5)
    _static(w, shape, sigma, False, "CS", n, u)


def test_fields_static_rejects_lattices_beyond_its_scratch(w):
    import torch
    nx = ny = 64
    nz = w.WDLB_STATIC_MAX_NODES // (nx * ny) + 1
    N = nx * ny * nz
    d = lambda k: torch.zeros(k * N, dtype=torch.float64, device="cuda")
    with pytest.raises(w.WDLBError) as ei:
        w.wdlb_fields_static((nx, ny, nz), 4.0, False, "CS", d(1), d(3), None, d(3), d(6))
    assert ei.value.status == 1
