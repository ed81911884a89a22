"""C ABI checks that need no GPU: the library builds and loads, exports every
function declared in include/wdlb.h, its host tables equal the oracle's
(rebuilt independently from the same rules), and invalid arguments are
rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wdlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wdlb_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_velocity_set_matches_oracle(lib, oracle_mod):
    c, w = lib.wdlb_velocity_set()
    co, wo = oracle_mod.velocities()
    lib_set = {tuple(v): wv for v, wv in zip(c.tolist(), w)}
    or_set = {tuple(v): wv for v, wv in zip(co.tolist(), wo)}
    assert lib_set.keys() == or_set.keys()
    for k in lib_set:
        assert lib_set[k] == pytest.approx(or_set[k], rel=1e-15)
    # library order: opposite directions adjacent
    for q in range(1, 19, 2):
        assert (c[q] == -c[q + 1]).all()


@pytest.mark.parametrize("sigma", [3.0, 4.0, 6.0, 8.0, 4.5])
def test_stencils_match_oracle(lib, oracle_mod, sigma):
    b, _ = lib.wdlb_stencil(sigma, 0)
    assert {tuple(v) for v in b.tolist()} == {tuple(v) for v in oracle_mod.ball(sigma).tolist()}
    e, w = lib.wdlb_stencil(sigma, 1)
    eo, wo = oracle_mod.shell(sigma)
    assert {tuple(v) for v in e.tolist()} == {tuple(v) for v in eo.tolist()}
    assert w == pytest.approx(wo, rel=1e-14)
    # +e/-e pairs are adjacent in the library's summation order
    assert (e[0::2] == -e[1::2]).all()


def test_compact_shell_matches_oracle(lib, oracle_mod):
    """The compact quadrature (two or three cubic orbits, weights from three
    moment conditions) is rebuilt independently on both sides: the same vectors
    at every sigma on a 0.05 grid, weights within the two solvers' rounding,
    and no shell where the oracle has none."""
    worst = 0.0
    for sigma in np.round(np.arange(1.0, 8.0001, 0.05), 2):
        ref = oracle_mod.shell_compact(float(sigma))
        if ref is None:
            with pytest.raises(lib.WDLBError):
                lib.wdlb_shell_table(float(sigma), "compact")
            continue
        e, w = lib.wdlb_shell_table(float(sigma), "compact")
        got = {tuple(v): x for v, x in zip(e.tolist(), w)}
        exp = {tuple(v): x for v, x in zip(ref[0].tolist(), ref[1])}
        assert got.keys() == exp.keys(), sigma
        worst = max(worst, max(abs(got[k] / exp[k] - 1) for k in got))
        assert (e[0::2] == -e[1::2]).all()
    assert worst < 1e-9
    e, w = lib.wdlb_shell_table(4.0, "full")
    assert len(e) == 210 and np.all(w == lib.wdlb_stencil(4.0, 1)[1])


def test_compact_rule_refused_where_it_has_no_shell(lib):
    so = lib.load_library()
    opt = lib.wdlb_options()
    so.wdlb_default_options(ctypes.byref(opt))
    opt.shell_rule = 1
    nb = ctypes.c_uint64()
    assert so.wdlb_workspace_size(lib.wdlb_lattice(8, 8, 8), 1.5, 0, ctypes.byref(opt), ctypes.byref(nb)) == 1
    assert so.wdlb_workspace_size(lib.wdlb_lattice(8, 8, 8), 4.0, 0, ctypes.byref(opt), ctypes.byref(nb)) == 0
    opt.shell_rule = 2
    assert so.wdlb_workspace_size(lib.wdlb_lattice(8, 8, 8), 4.0, 0, ctypes.byref(opt), ctypes.byref(nb)) == 1


def test_invalid_arguments_rejected(lib):
    so = lib.load_library()
    lat = lib.wdlb_lattice(8, 8, 41)
    opt = lib.wdlb_options()
    so.wdlb_default_options(ctypes.byref(opt))
    h = ctypes.c_void_p()
    g = (ctypes.c_double * 3)(0, 0, 0)
    assert so.wdlb_create(lat, 0.5, 1, 1.0, g, ctypes.byref(opt), ctypes.byref(h)) == 1     # sigma < 1
    assert so.wdlb_create(lat, 4.0, 1, 0.5, g, ctypes.byref(opt), ctypes.byref(h)) == 1     # tau <= 1/2
    assert so.wdlb_create(lib.wdlb_lattice(8, 8, 2), 4.0, 1, 1.0, g, ctypes.byref(opt), ctypes.byref(h)) == 1
    assert so.wdlb_create(lib.wdlb_lattice(0, 8, 8), 4.0, 0, 1.0, g, ctypes.byref(opt), ctypes.byref(h)) == 1
    opt.storage = 7
    assert so.wdlb_create(lat, 4.0, 1, 1.0, g, ctypes.byref(opt), ctypes.byref(h)) == 1
    assert not h.value
    assert "invalid" in lib.wdlb_last_error(None) or "tau" in lib.wdlb_last_error(None)
    assert so.wdlb_step(None, 1) == 1
    so.wdlb_destroy(None)   # NULL-safe


def test_workspace_size_scales_with_storage(lib):
    so = lib.load_library()
    lat = lib.wdlb_lattice(32, 32, 32)
    sizes = {}
    for name, code in lib.STORAGES.items():
        opt = lib.wdlb_options()
        so.wdlb_default_options(ctypes.byref(opt))
        opt.storage = code
        nb = ctypes.c_uint64()
        assert so.wdlb_workspace_size(lat, 4.0, 0, ctypes.byref(opt), ctypes.byref(nb)) == 0
        sizes[name] = nb.value
    N = 32 ** 3
    assert sizes["f64"] > sizes["f32"] > sizes["f16"]
    assert sizes["f32"] - sizes["f16"] >= 2 * 19 * N * 2 * 0.99


def test_fields_static_binding_checks_its_tensors():
    """The binding of wdlb_fields_static refuses, before any library call, a
    tensor of the wrong type, size or device: the C side cannot see a buffer's
    extent, and a wrong one would be read or written past its end."""
    torch = pytest.importorskip("torch")
    from paper_1304_7880_gb300 import wdlb as w
    lat = (4, 3, 5)
    N = 60
    bad = [
        (torch.zeros(N, dtype=torch.float32), torch.zeros(3 * N, dtype=torch.float64)),   # float32 n
        (torch.zeros(N, dtype=torch.float64), torch.zeros(3 * N - 1, dtype=torch.float64)),  # short u
        (torch.zeros(N, dtype=torch.float64), torch.zeros(3 * N, dtype=torch.float64)),   # host memory
    ]
    for d_n, d_u in bad:
        with pytest.raises(w.WDLBError) as ei:
            w.wdlb_fields_static(lat, 4.0, False, "CS", d_n, d_u, None, torch.zeros(3 * N, dtype=torch.float64),
                                 torch.zeros(6 * N, dtype=torch.float64))
        assert ei.value.status == 1
    with pytest.raises(w.WDLBError):
        w.wdlb_fields_static(lat, 4.0, False, "CS", None, None, None, None, None)
