"""Serving loop (continuous batching) on the GPU: requests submitted while
others are being stepped are admitted into the running batch, and each
result equals the same request solved alone with wdlb_run_steady (same
kernels, same residual cadence), also while sharing the device with a mix."""
import io
import json
import time

import numpy as np
import pytest

from paper_1304_7880_gb300 import synth

pytestmark = pytest.mark.gpu

# (lattice, sigma, n*, g_x, seed)
REQUESTS = [
    ((8, 8, 13), 3.0, 0.3, 1e-5, 51),
    ((16, 8, 17), 4.0, 0.4, 3e-6, 52),
    ((8, 8, 25), 4.0, 0.5, 1e-5, 53),
    ((12, 12, 21), 3.0, 0.45, 2e-6, 54),
    ((10, 8, 19), 4.0, 0.25, 5e-6, 55),
    ((12, 9, 27), 6.0, 0.3, 4e-6, 56),        # a third shell group (sigma 6) in the same batch
]
TOL = 1e-6


@pytest.fixture(scope="module")
def w():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_7880_gb300 import build, wdlb
    build.build()
    return wdlb


def test_server_results_equal_alone(w):
    srv = w.wdlb_server_create(128 << 20, max_active=8, check_every=100)
    ids = {}
    for k, (lat, sigma, nstar, gx, seed) in enumerate(REQUESTS):
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ids[w.wdlb_server_submit(srv, lat, sigma, True, 1.0, p["g"], n, u, tol=TOL, max_steps=200000,
                                 want_moments=True)] = k
        time.sleep(0.05 * k)          # later requests join a running batch
    results = {}
    t0 = time.time()
    while len(results) < len(ids) and time.time() - t0 < 300:
        for r in w.wdlb_server_poll(srv):
            results[ids[r["id"]]] = r
        time.sleep(0.01)
    info = w.wdlb_server_info(srv)
    w.wdlb_server_destroy(srv)
    assert len(results) == len(REQUESTS), info
    # the device time of the blocks of steps, a part of the server's clock
    assert 0 < info["gpu_step_s"] <= info["clock_s"], info
    for k, (lat, sigma, nstar, gx, seed) in enumerate(REQUESTS):
        r = results[k]
        assert r["status"] == 0 and r["residual"] < TOL
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ctx = w.wdlb_create(lat, sigma, True, 1.0, p["g"], storage="f32")
        w.wdlb_init_fields(ctx, n, u)
        steps, res = w.wdlb_run_steady(ctx, TOL, 100, 200000)
        n_a, u_a = w.wdlb_moments(ctx)
        st = w.wdlb_pore_average(ctx)
        w.wdlb_destroy(ctx)
        assert r["steps"] == steps
        assert np.array_equal(r["n"], n_a) and np.array_equal(r["u"], u_a)
        assert r["stats"]["flux_x"] == st["flux_x"]
        assert r["finish_s"] >= r["start_s"] >= r["submit_s"]


def test_server_compact_shell_results_equal_alone(w):
    """A server on the compact contact shell: sigma 3, 4 and 6 requests in one
    batch, each equal bit for bit to the request solved alone with that rule."""
    reqs = [REQUESTS[0], REQUESTS[2], REQUESTS[5]]
    srv = w.wdlb_server_create(64 << 20, max_active=4, check_every=100, shell_rule="compact")
    ids = {}
    for k, (lat, sigma, nstar, gx, seed) in enumerate(reqs):
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ids[w.wdlb_server_submit(srv, lat, sigma, True, 1.0, p["g"], n, u, tol=TOL, max_steps=200000,
                                 want_moments=True)] = k
    results = {}
    log = io.StringIO()              # one JSON line per finished solve
    t0 = time.time()
    while len(results) < len(ids) and time.time() - t0 < 300:
        for r in w.wdlb_server_poll(srv, log=log):
            results[ids[r["id"]]] = r
        time.sleep(0.01)
    w.wdlb_server_destroy(srv)
    assert len(results) == len(reqs)
    recs = [json.loads(line) for line in log.getvalue().splitlines()]
    assert sorted(r["id"] for r in recs) == sorted(ids)
    assert all(r["status"] == "OK" and r["mlups"] > 0 and r["latency_s"] >= r["run_s"] for r in recs)
    for k, (lat, sigma, nstar, gx, seed) in enumerate(reqs):
        r = results[k]
        assert r["status"] == 0 and r["residual"] < TOL
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ctx = w.wdlb_create(lat, sigma, True, 1.0, p["g"], storage="f32", shell_rule="compact")
        w.wdlb_init_fields(ctx, n, u)
        steps, _ = w.wdlb_run_steady(ctx, TOL, 100, 200000)
        n_a, u_a = w.wdlb_moments(ctx)
        w.wdlb_destroy(ctx)
        assert r["steps"] == steps
        assert np.array_equal(r["n"], n_a) and np.array_equal(r["u"], u_a)


def test_server_rejects_a_pore_larger_than_its_budget(w):
    srv = w.wdlb_server_create(4 << 20, max_active=2, check_every=100)
    p, n, u = synth.slit_poiseuille(32, 32, 65, 0.3, 4.0, 1.0, 1e-6, 7)
    rid = w.wdlb_server_submit(srv, (32, 32, 65), 4.0, True, 1.0, p["g"], n, u)
    out = []
    t0 = time.time()
    while not out and time.time() - t0 < 30:
        out = w.wdlb_server_poll(srv)
        time.sleep(0.01)
    w.wdlb_server_destroy(srv)
    assert out and out[0]["id"] == rid and out[0]["status"] == 2


def test_server_double_word_collision_results_equal_alone(w):
    """A server with the double-word collision (sigma 3, 4 and 6 requests in one
    batch, each its own tile kernel): every result equal bit for bit to the
    request solved alone with that collision."""
    reqs = [REQUESTS[0], REQUESTS[1], REQUESTS[5]]
    srv = w.wdlb_server_create(64 << 20, max_active=4, check_every=100, collision="dw")
    ids = {}
    for k, (lat, sigma, nstar, gx, seed) in enumerate(reqs):
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ids[w.wdlb_server_submit(srv, lat, sigma, True, 1.0, p["g"], n, u, tol=TOL, max_steps=200000,
                                 want_moments=True)] = k
    results = {}
    t0 = time.time()
    while len(results) < len(ids) and time.time() - t0 < 300:
        for r in w.wdlb_server_poll(srv):
            results[ids[r["id"]]] = r
        time.sleep(0.01)
    w.wdlb_server_destroy(srv)
    assert len(results) == len(reqs)
    for k, (lat, sigma, nstar, gx, seed) in enumerate(reqs):
        r = results[k]
        assert r["status"] == 0 and r["residual"] < TOL
        p, n, u = synth.slit_poiseuille(*lat, nstar, sigma, 1.0, gx, seed)
        ctx = w.wdlb_create(lat, sigma, True, 1.0, p["g"], storage="f32", collision="dw")
        w.wdlb_init_fields(ctx, n, u)
        steps, _ = w.wdlb_run_steady(ctx, TOL, 100, 200000)
        n_a, u_a = w.wdlb_moments(ctx)
        w.wdlb_destroy(ctx)
        assert r["steps"] == steps
        assert np.array_equal(r["n"], n_a) and np.array_equal(r["u"], u_a)
