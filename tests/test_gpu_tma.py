"""TMA staging of the tiled shell kernel's field tile (sigma 4: one
cp.async.bulk.tensor box for nu and one for hb per interior brick, behind an
mbarrier) against the per-node cp.async staging.  The two load the same tile,
so the populations must agree bit for bit, on every tile shape, in bulk and
in slits (where the box reads zeros beyond the walls and the kernel writes the
n = 0 state there), for both shell rules and both FP32 and FP16 storage.  The
give-up path of the bounded wait is driven by a barrier that nothing completes
(no copy issued) and must come back as WDLB_ERR_TIMEOUT."""
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


def _run(w, lat, walls, storage, rule, tile, staging, steps=12):
    nx, ny, nz = lat
    if walls:
        p, n, u = synth.slit_poiseuille(nx, ny, nz, 0.45, 4.0, 1.0, 1e-5, 21)
    else:
        n, u = synth.uniform_with_noise(nx, ny, nz, 0.45 / 64, 2e-2, 21, False)
    ctx = w.wdlb_create(lat, 4.0, walls, 1.0, (1e-5, 0.0, 0.0), storage=storage, shell_rule=rule, tile=tile,
                        autotune=False, staging=staging)
    w.wdlb_init_fields(ctx, n, u)
    w.wdlb_step(ctx, steps)
    w.wdlb_moments(ctx)                   # raises on any status bit
    out = w.wdlb_get_populations(ctx), w.wdlb_staging_info(ctx)
    w.wdlb_destroy(ctx)
    return out


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("walls,lat", [(False, (32, 24, 24)), (True, (24, 32, 30))])
def test_tma_tile_equals_cp_async_tile(w, walls, lat, tile):
    a, tma = _run(w, lat, walls, "f32", "full", tile, "auto")
    b, cpa = _run(w, lat, walls, "f32", "full", tile, "cp_async")
    assert tma and not cpa
    assert np.array_equal(a, b)


@pytest.mark.parametrize("storage,rule", [("f32", "compact"), ("f16", "full")])
def test_tma_tile_other_paths(w, storage, rule):
    lat = (32, 32, 37)
    walls = storage != "f16"        # FP16 storage is for periodic boxes only
    a, tma = _run(w, lat, walls, storage, rule, 2, "auto")
    b, _ = _run(w, lat, walls, storage, rule, 2, "cp_async")
    assert tma and np.array_equal(a, b)


def test_tma_not_used_where_rows_are_not_16_bytes(w):
    # nx = 30: the hb rows are 120 bytes, not a multiple of 16; sigma 3: a halo
    # of 3 puts the tile's first x off the 16-byte grid
    _, tma = _run(w, (30, 24, 24), False, "f32", "full", 2, "auto", steps=2)
    assert not tma
    ctx = w.wdlb_create((32, 24, 24), 3.0, False, 1.0, (0.0, 0.0, 0.0), storage="f32", autotune=False)
    assert not w.wdlb_staging_info(ctx)
    w.wdlb_destroy(ctx)


def test_tma_wait_that_runs_out_is_reported(w):
    """A wait on a barrier that nothing completes gives up after its poll
    budget: the brick is skipped, the status word carries the timeout, and the
    call reports WDLB_ERR_TIMEOUT instead of hanging."""
    lat = (32, 32, 32)
    n, u = synth.uniform_with_noise(*lat, 0.45 / 64, 2e-2, 3, False)
    ctx = w.wdlb_create(lat, 4.0, False, 1.0, (0.0, 0.0, 0.0), storage="f32", tile=2, autotune=False,
                        wait_limit=-64)
    assert w.wdlb_staging_info(ctx)
    w.wdlb_init_fields(ctx, n, u)
    w.wdlb_step(ctx, 1)
    with pytest.raises(w.WDLBError) as ei:
        w.wdlb_moments(ctx)
    assert ei.value.status == 5
    w.wdlb_destroy(ctx)
