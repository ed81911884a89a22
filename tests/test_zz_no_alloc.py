"""wdlb_fields_static, the entry point that allocates no device memory (for
callers running inside another framework's memory pool or a host that forbids
cudaMalloc), against the allocating entry point wdlb_fields on the same state.

wdlb_fields of a freshly initialised FP32 context (g = 0) evaluates the fields
with the neighbours' velocity equal to the initial u, which is what
wdlb_fields_static evaluates from device arrays n and u.  Both run FP32
arithmetic; the bound is the FP32 tolerance of the parity tests, 1e-5 of the
largest magnitude.  Two calls in a row, on two different states, check that the
shared scratch array carries nothing from one call to the next."""
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


@pytest.mark.parametrize("walls,shape", [(False, (24, 20, 16)), (True, (33, 16, 16))])
def test_fields_static_matches_fields(w, walls, shape):
    import torch
    sigma = 4.0
    nz, ny, nx = shape
    mask = np.ones(shape, dtype=bool)
    if walls:
        mask[0] = mask[-1] = False
    out_nb = torch.empty(shape, dtype=torch.float64, device="cuda")
    out_C = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    out_A = torch.empty((6,) + shape, dtype=torch.float64, device="cuda")
    for call, seed in enumerate((11, 12)):
        n, u = _state(shape, sigma, walls, seed)
        ctx = w.wdlb_create((nx, ny, nz), sigma, walls, 1.0, (0.0, 0.0, 0.0), storage="f32")
        w.wdlb_init_fields(ctx, n, u)
        nb_ref, C_ref, A_ref, _ = w.wdlb_fields(ctx)
        d_n = torch.from_numpy(n).cuda()
        d_u = torch.from_numpy(u).cuda()
        torch.cuda.synchronize()
        w.wdlb_fields_static((nx, ny, nz), sigma, walls, "CS", d_n, d_u, out_nb, out_C, out_A)
        torch.cuda.synchronize()
        nb, C, A = out_nb.cpu().numpy(), out_C.cpu().numpy(), out_A.cpu().numpy()
        np.testing.assert_allclose(nb[mask], nb_ref[mask], rtol=TOL)
        np.testing.assert_allclose(C[:, mask], C_ref[:, mask], rtol=0, atol=TOL * np.abs(C_ref[:, mask]).max())
        np.testing.assert_allclose(A[:, mask], A_ref[:, mask], rtol=0, atol=TOL * np.abs(A_ref[:, mask]).max())
        if walls:
            assert not C[:, ~mask].any() and not A[:, ~mask].any()
        w.wdlb_destroy(ctx)


def test_fields_static_rejects_lattices_beyond_its_scratch(w):
    import torch
    nx = ny = 64
    nz = w.WDLB_STATIC_MAX_NODES // (nx * ny) + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(w.WDLBError) as ei:
        w.wdlb_fields_static((nx, ny, nz), 4.0, False, "CS", d, d, None, d, d)
    assert ei.value.status == 1
