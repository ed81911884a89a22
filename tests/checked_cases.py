"""Cases for the bounds-checked build (run as a child process by
test_gpu_checked.py): every kernel variant of the time step on small ragged
lattices.  The library is the one WDLB_LIBRARY names (the checked or the
normal build).  Every case steps a few times and reads its moments, which
raises if a kernel index left its array; the populations of every case are
written to the .npz file given as the only argument, for a bitwise comparison
of the two builds."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1304_7880_gb300 import synth  # noqa: E402
from paper_1304_7880_gb300 import wdlb as w  # noqa: E402

# name: (lattice, sigma, walls, storage, shell rule, tile)
CASES = {
    "s3_periodic_t%d": ((13, 11, 19), 3.0, False, "f32", "full"),
    "s4_slit_t%d": ((10, 8, 27), 4.0, True, "f32", "full"),
    "s6_slit_t%d": ((12, 9, 35), 6.0, True, "f32", "full"),
    "s4_periodic_compact_t%d": ((17, 9, 12), 4.0, False, "f32", "compact"),
    "s6_slit_compact_t%d": ((12, 9, 35), 6.0, True, "f32", "compact"),
}
SINGLE = {
    "s4_bulk_f16": ((12, 8, 27), 4.0, False, "f16", "full"),
    "s4_slit_f64": ((10, 8, 27), 4.0, True, "f64", "full"),
    "s3.5_slit_compact": ((11, 9, 15), 3.5, True, "f32", "compact"),
    "s8_bulk_compact": ((16, 16, 20), 8.0, False, "f32", "compact"),
    "narrow_pore_s4": ((6, 5, 21), 4.0, True, "f32", "full"),
}
# the double-word collision (slits only): tiled kernels on every tile shape and
# the generic kernel (sigma 3.5, and a pore too narrow for the tiled kernel)
DW_CASES = {
    "s4_slit_dw_t%d": ((10, 8, 27), 4.0, True, "f32", "full"),
    "s6_slit_compact_dw_t%d": ((12, 9, 35), 6.0, True, "f32", "compact"),
}
DW_SINGLE = {
    "s3.5_slit_dw": ((11, 9, 15), 3.5, True, "f32", "full"),
    "narrow_pore_s4_dw": ((6, 5, 21), 4.0, True, "f32", "full"),
}


def state(lat, sigma, walls, seed):
    nx, ny, nz = lat
    return synth.uniform_with_noise(nx, ny, nz, 0.4 / sigma ** 3, 2e-2, seed, walls)


def run_case(lat, sigma, walls, storage, rule, tile, collision="fp32"):
    n, u = state(lat, sigma, walls, 7)
    ctx = w.wdlb_create(lat, sigma, walls, 1.0, (1e-5, 0.0, 0.0), storage=storage, shell_rule=rule, tile=tile,
                        autotune=False, collision=collision)
    w.wdlb_init_fields(ctx, n, u)
    w.wdlb_step(ctx, 5)
    w.wdlb_moments(ctx)          # raises on the checked build's bounds flag
    f = w.wdlb_get_populations(ctx)
    w.wdlb_destroy(ctx)
    return f


def main(out):
    res = {}
    for name, (lat, sigma, walls, storage, rule) in CASES.items():
        for tile in (0, 1, 2):
            res[name % tile] = run_case(lat, sigma, walls, storage, rule, tile)
    for name, (lat, sigma, walls, storage, rule) in SINGLE.items():
        res[name] = run_case(lat, sigma, walls, storage, rule, -1)
    for name, (lat, sigma, walls, storage, rule) in DW_CASES.items():
        for tile in (0, 1, 2):
            res[name % tile] = run_case(lat, sigma, walls, storage, rule, tile, "dw")
    for name, (lat, sigma, walls, storage, rule) in DW_SINGLE.items():
        res[name] = run_case(lat, sigma, walls, storage, rule, -1, "dw")
    # a batch of pores with different kernels (tiled sigma 3 and 4, generic narrow pore)
    b = w.wdlb_batch_create(4, 64 << 20, storage="f32")
    slots = []
    for lat, sigma in (((16, 16, 25), 4.0), ((12, 10, 19), 3.0), ((6, 5, 21), 4.0)):
        n, u = state(lat, sigma, True, 9)
        slots.append(w.wdlb_batch_add(b, lat, sigma, True, 1.0, (1e-5, 0.0, 0.0), n, u))
    w.wdlb_batch_step(b, 5)
    _, status = w.wdlb_batch_residuals(b, 5)
    assert all(s == 0 for s in np.asarray(status)[slots]), status
    for k, s in enumerate(slots):
        res["batch_%d" % k] = w.wdlb_get_populations(w.wdlb_batch_context(b, s))
    w.wdlb_batch_destroy(b)
    # the fields pass (FP64, generic kernel)
    n, u = state((9, 8, 7), 3.0, False, 11)
    ctx = w.wdlb_create((9, 8, 7), 3.0, False, 0.9, (1e-5, 0.0, 0.0), storage="f64")
    w.wdlb_init_fields(ctx, n, u)
    nbar, C, A, _ = w.wdlb_fields(ctx)
    w.wdlb_moments(ctx)
    res["fields_C"] = C
    res["fields_A"] = A
    w.wdlb_destroy(ctx)
    # the entry point without device allocation (generic kernels, sigma 8 with walls)
    import torch
    lat = (9, 8, 14)
    n, u = state(lat, 8.0, True, 13)
    d_n, d_u = torch.from_numpy(n).cuda(), torch.from_numpy(u).cuda()
    outs = [torch.empty(k * n.size, dtype=torch.float64, device="cuda") for k in (1, 3, 6)]
    w.wdlb_fields_static(lat, 8.0, True, "PY", d_n, d_u, *outs)   # raises on the bounds flag
    torch.cuda.synchronize()
    res["static_nbar"], res["static_C"], res["static_A"] = (t.cpu().numpy() for t in outs)
    np.savez(out, **res)
    print("checked cases: %d arrays, library %s" % (len(res), os.path.basename(w.LIB_PATH)))


if __name__ == "__main__":
    main(sys.argv[1])
