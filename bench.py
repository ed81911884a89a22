#!/usr/bin/env python3
"""Benchmark of the WDLB lattice update on GB300.

Headline workload: 64 slit pores in one batch (widths H uniform in [3 sigma,
30 sigma] at sigma = 4, i.e. 13-121 z-nodes, x-y 32 x 32, n* uniform in
[0.1, 0.57], g_x log-uniform in [1e-7, 1e-5], tau = 1), FP32 deviation storage
with FP64 reductions.  One benchmark step = 100 lattice time steps of every
pore (each: moments and field velocity, smeared density, shell sums +
collision + streaming; one launch per phase for all pores, replayed from a
CUDA graph) followed by the FP64 steady-state residual of every pore.  Metric:
MLUPS (lattice-node updates per second).  Further legs: the 128^3 bulk box
(FP32, FP16, FP64, compact shell), the 256 x 256 x 161 slit, serving, the
viscosity sweeps, and the FP64 oracle on the host cores.

  python bench.py [--gpus N --steps K --warmup W]      this library (C ABI)
  python bench.py --impl reference ...                 the FP64 CPU oracle

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of the
batch (the workload has no exchange step): weak scaling, no collective on the
data path; the elapsed time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (lattice-node updates/s) & HBM roofline frac, batched FP32 vs plain FP64; p50/p99 solve"
UNIT = "MLUPS"
L = 128
SIGMA = 4.0                    # sigma of the 128^3 box legs (--sigma)
BATCH_SIGMA = 4.0              # sigma of the batched pores
SUB = 100                      # lattice time steps per benchmark step
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
BATCH_WORKLOAD = ("64 slit pores 32x32x(13..121) (H uniform in [3 sigma, 30 sigma]), sigma=4 lattice units, "
                  "walls z=0 and z=nz-1, n* uniform in [0.1, 0.57] (below the scheme's stability limit in slits), "
                  "g_x log-uniform in [1e-7, 1e-5], tau=1, D3Q19, Carnahan-Starling contact value, K=2, "
                  "seeded 1e-3 density noise")
WORKLOAD = ("bulk periodic box 128^3, sigma=4 lattice units, packing fraction 0.3, D3Q19, "
            "Carnahan-Starling contact value, K=2, tau=1, shear wave u_x=1e-4 sin(2 pi z/128), 1e-4 density noise")


def shell_size(sigma):
    R = int(math.floor(sigma + 0.5))
    c = 0
    for x in range(-R, R + 1):
        for y in range(-R, R + 1):
            for z in range(-R, R + 1):
                r2 = x * x + y * y + z * z
                if (sigma - 0.5) ** 2 < r2 <= (sigma + 0.5) ** 2:
                    c += 1
    return c


# Algorithmic FP32 operations per node update of the shell + collide kernel
# (an FMA counts 2): per shell vector 52 (contact value 9, velocity
# difference 3, khat.dv and q khat.dv 6, the F^mf, F^viscous and A sums 36,
# t 1), plus 475 for moments, collision and the force terms.
FLOPS_PER_PAIR = 52
# the compact shell's per-vector weight: three more multiplies per (+e, -e) pair
FLOPS_PER_PAIR_WEIGHTED = FLOPS_PER_PAIR + 1.5
FLOPS_COLLIDE = 475
# Algorithmic HBM bytes per node update: read and write 19 populations.
BYTES_PER_NODE = {"f64": 19 * 2 * 8, "f32": 19 * 2 * 4, "f16": 19 * 2 * 2}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash():
    """Hash of the files that define the step kernels' device code and of the
    build flags (host-side launch code does not change a kernel's traffic)."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1304_7880_gb300")
    for f in ("csrc/wdlb_common.cuh", "csrc/wdlb_dw.cuh", "csrc/wdlb_kernels.cuh", "csrc/wdlb_shell_tiled.cuh",
              "csrc/wdlb_step_kernels.cuh", "build.py"):
        with open(os.path.join(pkg, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_shell_tiled_batch64_traffic.txt")
STEP_BYTES_FILE = os.path.join(ROOT, "profiles", "step_bulk128_dram_record.txt")


def _record(path):
    rec = {}
    try:
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
    except OSError:
        pass
    return rec


def recorded_step_bytes(rule):
    """Measured DRAM bytes per node update of the whole FP32 128^3 step (moments,
    smeared density and shell kernels) with the given shell rule, from the
    committed ncu record, used only if taken on the current kernel sources."""
    rec = _record(STEP_BYTES_FILE)
    try:
        if rec.get("source_hash") == kernel_source_hash():
            return float(rec["bytes_per_node_" + rule])
    except (KeyError, ValueError):
        pass
    return None


def recorded_traffic(nodes):
    """DRAM bytes per launch of the batch's shell kernel from the committed ncu
    summary (lines "key: value"), used only if it was taken on the current
    kernel sources and a workload of the same node count."""
    try:
        rec = {}
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("source_hash") == kernel_source_hash() and int(rec.get("nodes", -1)) == nodes:
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class RankSync:
    """Barrier and maximum over the ranks of a torchrun job (one replica per
    GPU; no collective on the data path).  dist is torch.distributed with an
    initialised process group, or None for one process; device is where the
    reduction tensor lives (cuda for NCCL, cpu for gloo)."""

    def __init__(self, dist, device):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def job_mlups(world, nodes, time_steps, seconds):
    """Whole-job throughput of `world` replicas that each updated `nodes`
    lattice nodes `time_steps` times in `seconds` (the slowest rank's time)."""
    return world * nodes * time_steps / seconds / 1e6


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(conn, pore_index, count, seed):
    """One host process stepping one pore of the batched workload with the
    oracle, on command ("step", k) -> replies the nodes updated."""
    import oracle
    from paper_1304_7880_gb300 import synth
    pp, n, u = synth.batched_pores(count=count, seed=seed)[pore_index]
    o = oracle.Oracle(pp["nx"], pp["ny"], pp["nz"], pp["walls"], pp["sigma"], pp["tau"], pp["g"])
    o.init(n, u)
    nodes = pp["nx"] * pp["ny"] * pp["nz"]
    conn.send(("ready", nodes))
    while True:
        msg = conn.recv()
        if msg[0] == "stop":
            break
        o.step(int(msg[1]))
        conn.send(("done", nodes * int(msg[1])))
    conn.close()


class OraclePool:
    """`procs` host processes (started with spawn, never forked from a process
    that holds a CUDA context), each holding one pore of the batched workload
    in the oracle.  step(k) runs k time steps of every pore concurrently and
    returns the lattice-node updates done."""

    def __init__(self, procs, count=64, seed=4):
        import multiprocessing as mp
        import oracle
        oracle.build()                 # once, before the workers load it
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for k in range(procs):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, k % count, count, seed), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        self.nodes = [c.recv()[1] for c in self.conns]

    def step(self, k):
        for c in self.conns:
            c.send(("step", k))
        return sum(c.recv()[1] for c in self.conns)

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_oracle():
    """The FP64 oracle as it stands, on bounded samples of the batched
    workload: one pore on one host thread, then one pore per host core
    stepped concurrently (independent processes)."""
    model = cpu_model()
    one = OraclePool(1)
    t0 = time.perf_counter()
    done = one.step(2)
    dt1 = time.perf_counter() - t0
    one.close()
    cores = host_cores()
    pool = OraclePool(cores)
    pool.step(1)                       # warm-up
    t0 = time.perf_counter()
    done_all = pool.step(2)
    dt_all = time.perf_counter() - t0
    pool.close()
    return {"value": done_all / dt_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": "2 time steps of %d pores of the 64-pore batch, one pore per host core in its own process "
                      "(%d nodes, %.1f s)" % (cores, sum(pool.nodes), dt_all),
            "single_thread": {"value": done / dt1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": "2 time steps of pore 0 of the batch (%d nodes, %.1f s)" % (done // 2, dt1)}}


def run_serving(w, synth, np, rate, window_s, drain_s, max_active=48, tol=1e-8, collision="fp32"):
    """Continuous-batching server fed with Poisson arrivals in real time; each
    request runs until the relative change per step of its pore flux is below
    tol.  Requests arrive for window_s seconds, then the server drains for up
    to drain_s seconds; latency = finish - submit.  The fields are generated
    before the clock starts, so submission keeps pace with the arrivals."""
    reqs = synth.serving_requests(rate, window_s)
    fields = [synth.slit_poiseuille(q["nx"], q["ny"], q["nz"], q["n_star"], q["sigma"], q["tau"], q["gx"], seed)
              for _, q, seed in reqs]
    srv = w.wdlb_server_create(24 << 30, max_active=max_active, check_every=100, collision=collision)
    submitted = {}
    t_start = time.perf_counter()
    for (t_arr, q, _), (pp, n, _) in zip(reqs, fields):
        now = time.perf_counter() - t_start
        if t_arr > now:
            time.sleep(t_arr - now)
        rid = w.wdlb_server_submit(srv, (q["nx"], q["ny"], q["nz"]), q["sigma"], True, q["tau"], pp["g"], n,
                                   tol=tol, max_steps=10 ** 6)
        submitted[rid] = q
    del fields
    done = []
    while time.perf_counter() - t_start < window_s + drain_s:
        done.extend(w.wdlb_server_poll(srv))
        if len(done) == len(submitted):
            break
        time.sleep(0.02)
    elapsed = time.perf_counter() - t_start
    done.extend(w.wdlb_server_poll(srv))
    info = w.wdlb_server_info(srv)
    w.wdlb_server_destroy(srv)
    ok = [r for r in done if r["status"] == 0]
    by_status = {}
    for r in done:
        name = w.STATUS_NAMES.get(r["status"], str(r["status"]))
        by_status[name] = by_status.get(name, 0) + 1
    failed = [{"id": r["id"], "status": w.STATUS_NAMES.get(r["status"], str(r["status"])), "steps": r["steps"],
               "residual": r["residual"], "sigma": submitted[r["id"]]["sigma"],
               "H": submitted[r["id"]]["nz"] - 2, "nxy": submitted[r["id"]]["nx"],
               "n_star": round(submitted[r["id"]]["n_star"], 4), "g_x": submitted[r["id"]]["gx"]}
              for r in done if r["status"] != 0]
    lat = np.array([r["finish_s"] - r["submit_s"] for r in ok]) if ok else np.array([np.nan])
    node_steps = sum(submitted[r["id"]]["nx"] * submitted[r["id"]]["ny"] * submitted[r["id"]]["nz"] * r["steps"]
                     for r in ok)
    return {"offered_rate_per_s": round(rate, 3), "arrival_window_s": window_s, "submitted": len(submitted),
            "completed": len(ok), "failed": len(done) - len(ok), "by_status": by_status, "failed_requests": failed,
            "elapsed_s": round(elapsed, 3),
            "solves_per_s": len(ok) / elapsed, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "backlog_at_end": info["queued"] + info["active"],
            "completed_mlups": node_steps / elapsed / 1e6, "server_mlups": info["node_steps"] / elapsed / 1e6,
            "gpu_step_fraction": info["gpu_step_s"] / elapsed,
            "max_active": max_active, "collision": collision}


SERVE_WORKLOAD = ("slit Poiseuille requests: sigma in {3,4,6}, H/sigma lognormal (median 10, log-sd 0.5) clipped "
                  "to [3,60], x-y 16..64, n* in [0.1,0.57], g_x log-uniform [1e-7,1e-5], tau=1, FP32, steady "
                  "state at relative pore-flux change < 1e-8 per step (checked every 100 steps), 24 GiB "
                  "admission budget, FIFO admission, at most 48 pores stepped together")


def run_single_pore(w, synth, np, count=2, tol=1e-8):
    """The first `count` requests of the serving stream solved one at a time,
    alone on the GPU, on the plain FP64 path, the FP32 path (same kernels as
    the batch) and FP32 storage with the double-word collision, to the same
    steady-state tolerance; solves/s of each and the largest relative
    difference of each FP32 path's pore fluxes from the FP64 path's."""
    reqs = synth.serving_requests(200.0, 5.0)[:count]
    out = {}
    flux = {}
    for path in ("f64", "f32", "f32_dw"):
        storage, collision = ("f32", "dw") if path == "f32_dw" else (path, "fp32")
        t_total, steps_total = 0.0, 0
        for k, (_, q, seed) in enumerate(reqs):
            pp, n, _ = synth.slit_poiseuille(q["nx"], q["ny"], q["nz"], q["n_star"], q["sigma"], q["tau"], q["gx"],
                                             seed)
            ctx = w.wdlb_create((q["nx"], q["ny"], q["nz"]), q["sigma"], True, q["tau"], pp["g"], storage=storage,
                                collision=collision)
            w.wdlb_init_fields(ctx, n)
            t0 = time.perf_counter()
            steps, _ = w.wdlb_run_steady(ctx, tol, 100, 10 ** 6)
            t_total += time.perf_counter() - t0
            steps_total += steps
            flux[(path, k)] = w.wdlb_pore_average(ctx)["flux_x"]
            w.wdlb_destroy(ctx)
        out[path] = {"solves_per_s": count / t_total, "seconds": t_total, "time_steps": steps_total}
    for path in ("f32", "f32_dw"):
        out[path]["flux_rel_diff_max_vs_f64"] = max(abs(flux[(path, k)] - flux[("f64", k)]) / abs(flux[("f64", k)])
                                                   for k in range(count))
    out["sample"] = ("first %d requests of the serving stream, solved one at a time to relative pore-flux "
                     "change < %g per step" % (count, tol))
    return out


def run_serving_pair(w, synth, np):
    """Overload at 200 requests/s measures the capacity (completed solves/s);
    a second run offered 70 % of that capacity gives latencies with a bounded
    queue."""
    over = run_serving(w, synth, np, rate=200.0, window_s=5.0, drain_s=25.0)
    cap = over["solves_per_s"]
    out = {"workload": SERVE_WORKLOAD, "overload": over, "capacity_solves_per_s": cap}
    if cap > 0:
        out["at_70pct_capacity"] = run_serving(w, synth, np, rate=0.7 * cap, window_s=20.0, drain_s=20.0)
    # capacity of the served stream with the double-word collision (steady
    # flows within 1e-5 of the FP64 oracle on u_x and flux)
    out["overload_dw_collision"] = run_serving(w, synth, np, rate=200.0, window_s=5.0, drain_s=25.0, collision="dw")
    out["single_pore"] = run_single_pore(w, synth, np)
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host's cores, one
    pore of the batched workload per core in its own process; one benchmark
    step = one time step of every such pore."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    pool = OraclePool(cores)
    for _ in range(args.warmup):
        pool.step(1)
    done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        done += pool.step(1)
    dt = time.perf_counter() - t0
    nodes = sum(pool.nodes)
    pool.close()
    value = done / dt / 1e6
    sample = ("1 time step per benchmark step of %d of the batch's 64 pores (%d nodes), one pore per host core, "
              "each in its own process" % (cores, nodes))
    cfg = {"workload": BATCH_WORKLOAD, "sample": sample, "nodes": nodes,
           "parallelism": "%d host processes (%s)" % (cores, cpu_model())}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_box_only(args, w, synth, torch):
    """The 128^3 bulk box alone, device-resident (for profiling): warm-up, then
    `steps` benchmark steps of SUB time steps, and one instrumented pass."""
    p, n, u = synth.bulk_shear_128(sigma=SIGMA)
    ctx = w.wdlb_create((L, L, L), p["sigma"], False, p["tau"], p["g"], storage="f32", tile=args.tile,
                        shell_rule=args.shell_rule, interactions=bool(args.interactions))
    w.wdlb_init_fields_device(ctx, torch.from_numpy(n).cuda(), torch.from_numpy(u).cuda())
    for _ in range(args.warmup):
        w.wdlb_step(ctx, SUB)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(ctx.stream)
    for _ in range(args.steps):
        w.wdlb_step(ctx, SUB)
    b.record(ctx.stream)
    torch.cuda.synchronize()
    ms = w.wdlb_profile_step(ctx, SUB)
    print(json.dumps({"only_device": True, "workload": WORKLOAD, "shell_rule": args.shell_rule,
                      "value": L ** 3 * SUB * args.steps / (a.elapsed_time(b) * 1e-3) / 1e6, "unit": UNIT,
                      "kernels_ms": ms, "tile_shape": w.wdlb_tile_info(ctx)[1], "tma": w.wdlb_staging_info(ctx)}),
          flush=True)
    w.wdlb_destroy(ctx)
    return 0


def fp32_peak_tflops(sm_count, sm_mhz):
    """FP32 FMA issue peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    sync = RankSync(dist, "cuda")
    barrier = sync.barrier
    max_over_ranks = sync.max

    from paper_1304_7880_gb300 import build, synth
    if rank == 0:
        build.build()
    barrier()
    from paper_1304_7880_gb300 import wdlb as w

    if args.only_device and args.workload == "bulk128":
        return run_box_only(args, w, synth, torch)

    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    alu_peak = fp32_peak_tflops(sm_count, SM_MAX_MHZ_NOMINAL)
    peaks, peak_kind = measured_peaks()

    # ---------------- headline: the 64-pore batch, device-resident ----------------
    pores = synth.batched_pores(seed=4 + rank, sigma=BATCH_SIGMA)
    nodes_b = sum(pp["nx"] * pp["ny"] * pp["nz"] for pp, _, _ in pores)
    probe = w.wdlb_batch_create(1, 1 << 20, storage="f32")
    pool = 0
    for pp, _, _ in pores:
        pool += (w.wdlb_batch_pore_bytes(probe, (pp["nx"], pp["ny"], pp["nz"]), pp["sigma"], pp["walls"]) + 255) // 256 * 256
    w.wdlb_batch_destroy(probe)
    # the built-in tile rule (sigma 4: 8 x 8 x 4 bricks at every pore height)
    # keeps the shell phase one launch for all pores
    bt = w.wdlb_batch_create(len(pores), pool + (1 << 20), storage="f32", autotune=False,
                             collision=args.collision if args.only_device else "fp32")
    slots = [w.wdlb_batch_add(bt, (pp["nx"], pp["ny"], pp["nz"]), pp["sigma"], pp["walls"], pp["tau"], pp["g"], nn, uu)
             for pp, nn, uu in pores]
    tiles = sorted({w.wdlb_tile_info(w.wdlb_batch_context(bt, s)) for s in slots})
    tma_pores = sum(w.wdlb_staging_info(w.wdlb_batch_context(bt, s)) for s in slots)

    def batch_bench_step():
        w.wdlb_batch_step(bt, SUB)
        return w.wdlb_batch_residuals(bt, SUB)

    for _ in range(args.warmup):
        batch_bench_step()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    launches0 = w.wdlb_batch_launch_count(bt)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(bt.stream)
    for _ in range(args.steps):
        batch_bench_step()
    ev1.record(bt.stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if rank == 0 else None
    gpu_launches = w.wdlb_batch_launch_count(bt) - launches0
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1))
    value = job_mlups(world, nodes_b, SUB * args.steps, elapsed_ms * 1e-3)
    res, st = w.wdlb_batch_residuals(bt, SUB)
    assert all(int(st[s]) == 0 for s in slots), st
    # per-kernel durations for the roofline: the same batch stepped phase by
    # phase with CUDA events around each launch on the batch stream
    prof_steps = max(1, min(args.steps, 5))
    kms = [0.0, 0.0, 0.0]
    torch.cuda.synchronize()
    ia = torch.cuda.Event(enable_timing=True)
    ib = torch.cuda.Event(enable_timing=True)
    ia.record(bt.stream)
    for _ in range(prof_steps):
        ms = w.wdlb_batch_profile_step(bt, SUB)
        for k in range(3):
            kms[k] += ms[k] / prof_steps
    ib.record(bt.stream)
    torch.cuda.synchronize()
    instrumented_ms = max_over_ranks(ia.elapsed_time(ib)) / prof_steps
    w.wdlb_batch_destroy(bt)

    if args.only_device:
        if rank == 0:
            print(json.dumps({"only_device": True, "value": value, "unit": UNIT, "ms_per_step": elapsed_ms / args.steps,
                              "time_steps_per_step": SUB, "kernels_ms": kms, "instrumented_ms_per_step": instrumented_ms,
                              "gpu_launches": int(gpu_launches), "tiles": tiles}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---------------- the same batch on other forms of the step ----------------
    def batch_leg(persistent, collision, form):
        bp = w.wdlb_batch_create(len(pores), pool + (1 << 20), storage="f32", autotune=False, persistent=persistent,
                                 collision=collision)
        pslots = [w.wdlb_batch_add(bp, (pp["nx"], pp["ny"], pp["nz"]), pp["sigma"], pp["walls"], pp["tau"], pp["g"],
                                   nn, uu) for pp, nn, uu in pores]
        for _ in range(args.warmup):
            w.wdlb_batch_step(bp, SUB)
            w.wdlb_batch_residuals(bp, SUB)
        pa = torch.cuda.Event(enable_timing=True)
        pb = torch.cuda.Event(enable_timing=True)
        pl0 = w.wdlb_batch_launch_count(bp)
        torch.cuda.synchronize()
        pa.record(bp.stream)
        for _ in range(args.steps):
            w.wdlb_batch_step(bp, SUB)
            w.wdlb_batch_residuals(bp, SUB)
        pb.record(bp.stream)
        torch.cuda.synchronize()
        _, pst = w.wdlb_batch_residuals(bp, SUB)
        p_ms = max_over_ranks(pa.elapsed_time(pb))
        leg = {"value": job_mlups(world, nodes_b, SUB * args.steps, p_ms * 1e-3), "unit": UNIT,
               "ms_per_step": p_ms / args.steps, "gpu_launches": w.wdlb_batch_launch_count(bp) - pl0,
               "status_ok": all(int(pst[s]) == 0 for s in pslots), "form": form}
        w.wdlb_batch_destroy(bp)
        return leg

    persistent_leg = batch_leg(True, "fp32", "one persistent kernel per %d time steps; each pore's phases follow one "
                                             "another without device-wide barriers (value: graph replays of one "
                                             "launch per phase)" % SUB)
    dw_leg = batch_leg(False, "dw", "double-word collision (WDLB_COLLISION_DW): the collision and the push's "
                                    "re-encoding in pairs of floats, FP32 storage; steady slit flows within 1e-5 of "
                                    "the FP64 oracle on u_x and flux, as with the FP32 collision and its in-plane "
                                    "momentum correction")

    # ---------------- end to end through the public batch API and host buffers ----------------
    pin = []
    for pp, nn, uu in pores:
        a = torch.empty(nn.shape, dtype=torch.float64, pin_memory=True)
        b = torch.empty(uu.shape, dtype=torch.float64, pin_memory=True)
        a.copy_(torch.from_numpy(nn))
        b.copy_(torch.from_numpy(uu))
        on = torch.empty(nn.shape, dtype=torch.float64, pin_memory=True)
        ou = torch.empty(uu.shape, dtype=torch.float64, pin_memory=True)
        pin.append((pp, a.numpy(), b.numpy(), on.numpy(), ou.numpy()))
    h2d = sum(a.nbytes + b.nbytes for _, a, b, _, _ in pin)
    d2h = sum(a.nbytes + b.nbytes for _, _, _, a, b in pin)
    # two batches, each on its own stream: while one steps, the next step's
    # pores are admitted into the other (their host-to-device copies and init
    # kernels overlap the time steps), and the finished batch's results are
    # read back after its steps; every copy stays inside the timed region,
    # pipeline fill and drain included
    be = [w.wdlb_batch_create(len(pores), pool + (1 << 20), storage="f32", autotune=False) for _ in range(2)]

    def admit(b):
        return [w.wdlb_batch_add(b, (pp["nx"], pp["ny"], pp["nz"]), pp["sigma"], pp["walls"], pp["tau"], pp["g"], a, u)
                for pp, a, u, _, _ in pin]

    def finish(b, ss):
        for s, (_, _, _, on, ou) in zip(ss, pin):
            w.wdlb_moments(w.wdlb_batch_context(b, s), on, ou)
        for s in ss:
            w.wdlb_batch_remove(b, s)

    def e2e_run(k, pipelined):
        if not pipelined:
            for _ in range(k):
                ss = admit(be[0])
                w.wdlb_batch_step(be[0], SUB)
                finish(be[0], ss)
            return
        cur, nxt = be
        ss = admit(cur)
        w.wdlb_batch_step(cur, SUB)
        for _ in range(k - 1):
            ss_next = admit(nxt)
            w.wdlb_batch_step(nxt, SUB)
            finish(cur, ss)
            cur, nxt, ss = nxt, cur, ss_next
        finish(cur, ss)

    e2e_steps = max(4, args.steps // 2)
    e2e_vals = {}
    for form in (False, True):
        e2e_run(2, form)
        barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps, form)
        e2e_vals[form] = job_mlups(world, nodes_b, SUB * e2e_steps, max_over_ranks(time.perf_counter() - t0))
        barrier()
        assert all(np.isfinite(on).all() for _, _, _, on, _ in pin)
    for b in be:
        w.wdlb_batch_destroy(b)
    e2e_value = e2e_vals[True]

    # ---------------- the 128^3 bulk box (device-resident) ----------------
    p, n_h, u_h = synth.bulk_shear_128(seed=2 + rank, sigma=SIGMA)
    N = L ** 3
    shape = (p["nx"], p["ny"], p["nz"])

    def make(storage, shell_rule="full"):
        ctx = w.wdlb_create(shape, p["sigma"], p["walls"], p["tau"], p["g"], storage=storage, tile=args.tile,
                            shell_rule=shell_rule)
        d_n = torch.from_numpy(n_h).cuda()
        d_u = torch.from_numpy(u_h).cuda()
        torch.cuda.synchronize()
        w.wdlb_init_fields_device(ctx, d_n, d_u)
        ctx.stream.synchronize()
        return ctx

    def box_leg(storage, rule, sub, reps):
        c2 = make(storage, rule)
        w.wdlb_step(c2, sub)
        pk = [0.0, 0.0, 0.0]
        for _ in range(reps):          # per-kernel durations (instrumented pass)
            ms = w.wdlb_profile_step(c2, sub)
            for k in range(3):
                pk[k] += ms[k] / reps
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(c2.stream)
        for _ in range(reps):          # throughput: the production path
            w.wdlb_step(c2, sub)
            w.wdlb_pore_average(c2)
        b.record(c2.stream)
        torch.cuda.synchronize()
        t = max_over_ranks(a.elapsed_time(b))
        mlups = job_mlups(world, N, sub * reps, t * 1e-3)
        out = {"value": mlups, "unit": UNIT, "kernels_ms": pk, "tile_shape": w.wdlb_tile_info(c2)[1],
               "hbm_frac_of_measured": mlups * 1e6 * BYTES_PER_NODE[storage] / 1e9 / peaks["hbm_gbs"]}
        if storage == "f32":
            measured = recorded_step_bytes(rule)
            out.update({"measured_bytes_per_node": measured,
                        "hbm_frac_from_measured_bytes": None if measured is None else
                        mlups * 1e6 * measured / 1e9 / peaks["hbm_gbs"]})
            ns = len(w.wdlb_shell_table(SIGMA, rule)[1]) if rule == "compact" else shell_size(SIGMA)
            fl = ns * (FLOPS_PER_PAIR_WEIGHTED if rule == "compact" else FLOPS_PER_PAIR) + FLOPS_COLLIDE
            tf = fl * N / (pk[2] * 1e-3) / 1e12
            out.update({"shell_vectors": ns, "flops_per_node": fl, "shell_kernel_alu_frac": tf / alu_peak,
                        "shell_kernel_tflops": tf,
                        "shell_kernel_hbm_frac_of_measured": BYTES_PER_NODE[storage] * N / (pk[2] * 1e-3)
                        / 1e9 / peaks["hbm_gbs"]})
        w.wdlb_destroy(c2)
        return out

    paths = {}
    for name, storage, rule, sub, reps in (("bulk128_f32", "f32", args.shell_rule, SUB, max(3, args.steps // 2)),
                                           ("bulk128_f32_compact_shell", "f32", "compact", SUB, 3),
                                           ("bulk128_f16", "f16", "full", SUB, 3),
                                           ("bulk128_f64", "f64", "full", 10, 2)):
        paths[name] = box_leg(storage, rule, sub, reps)

    # ---------------- the full-size slit 256 x 256 x 161 (FP32) ----------------
    sp, sn, su = synth.slit_poiseuille(256, 256, 161, 0.3, SIGMA, 0.8, 1e-6, seed=3)
    cs = w.wdlb_create((256, 256, 161), SIGMA, True, 0.8, sp["g"], storage="f32")
    w.wdlb_init_fields(cs, sn, su)
    w.wdlb_step(cs, 50)
    pk = w.wdlb_profile_step(cs, 20)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(cs.stream)
    w.wdlb_step(cs, 200)
    w.wdlb_pore_average(cs)
    b.record(cs.stream)
    torch.cuda.synchronize()
    Ns = 256 * 256 * 161
    paths["slit_256x256x161_f32"] = {"value": job_mlups(world, Ns, 200, max_over_ranks(a.elapsed_time(b)) * 1e-3),
                                     "unit": UNIT, "kernels_ms": pk, "tile_shape": w.wdlb_tile_info(cs)[1],
                                     "workload": "slit 256x256x161, walls z=0,160, sigma=4, n*=0.3, tau=0.8, "
                                                 "g_x=1e-6, FP32; 200 time steps + pore average"}
    w.wdlb_destroy(cs)

    # ---------------- serving: Poisson arrivals of steady-state slit solves ----------------
    serve = None
    if not args.no_serve:
        serve = run_serving_pair(w, synth, np)

    # ---------------- pore-viscosity sweep (Sec. 5, Fig. 2's experiment) ----------------
    sweep = None
    if not args.no_serve:
        from paper_1304_7880_gb300 import sweeps
        widths = [8, 12, 16, 24, 32, 48, 64, 96, 128, 160, 200]
        sweep = {"widths_H": widths, "sigma": 4.0, "tau": 1.0, "g_x": 1e-6,
                 "method": "steady slit Poiseuille per width through the serving loop (relative pore-flux change "
                           "< 1e-8 per step), eta_eff = <n> g H^2 / (12 <u_x>) over the long-wave bulk shear "
                           "viscosity at <n>"}
        t0 = time.perf_counter()
        for chi in (0.11, 0.32):
            res = sweeps.pore_viscosity_sweep(chi, widths)
            sweep["ratio_chi_%g" % chi] = [round(r["ratio"], 5) if r["status"] == 0 else None for r in res]
        dt = time.perf_counter() - t0
        t1 = time.perf_counter()
        cres_p = sweeps.pore_viscosity_sweep(0.11, widths, shell_rule="compact")
        sweep["ratio_chi_0.11_compact_shell"] = [round(r["ratio"], 5) if r["status"] == 0 else None for r in cres_p]
        sweep["compact_shell_seconds"] = time.perf_counter() - t1
        sweep["solves"] = 2 * len(widths)
        sweep["seconds"] = dt
        sweep["solves_per_s"] = 2 * len(widths) / dt
        t0 = time.perf_counter()
        bres = sweeps.bulk_viscosity_sweep([0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.35])
        sweep["bulk_sigma8"] = {"chi": [r["chi"] for r in bres if r["K"] == 2.0],
                                "eta_K2": [r["eta"] for r in bres if r["K"] == 2.0],
                                "eta_K0": [r["eta"] for r in bres if r["K"] == 0.0],
                                "measured_over_theory_K2": [round(r["eta"] / r["eta_theory"], 5)
                                                            for r in bres if r["K"] == 2.0],
                                "seconds": time.perf_counter() - t0}
        t0 = time.perf_counter()
        # the compact shell's density limit at sigma 8 lies between n* = 0.5 and 0.55 (chi 0.26-0.29)
        cres = sweeps.bulk_viscosity_sweep([0.05, 0.1, 0.15, 0.2, 0.25], shell_rule="compact")
        sweep["bulk_sigma8_compact_shell"] = {
            "chi": [r["chi"] for r in cres if r["K"] == 2.0],
            "eta_K2": [r["eta"] for r in cres if r["K"] == 2.0],
            "eta_K0": [r["eta"] for r in cres if r["K"] == 0.0],
            "measured_over_theory_K2": [round(r["eta"] / r["eta_theory"], 5) for r in cres if r["K"] == 2.0],
            "over_full_shell_K2": [round(c["eta"] / f["eta"], 5) for c, f in zip(cres, bres) if c["K"] == 2.0],
            "seconds": time.perf_counter() - t0}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---------------- roofline of the dominant kernel (the batch's shell phase) ----------------
    nshell = shell_size(BATCH_SIGMA)
    flops_per_node = nshell * FLOPS_PER_PAIR + FLOPS_COLLIDE
    shell_ms = kms[2]
    achieved_tflops = flops_per_node * nodes_b / (shell_ms * 1e-3) / 1e12
    step_ms = sum(kms)
    hbm_achieved = BYTES_PER_NODE["f32"] * nodes_b / (step_ms * 1e-3) / 1e9
    kname = ", ".join("k_step_shell_tiled<float, %d, %d, true, false>" % (int(round(2 * BATCH_SIGMA)), t[1]) if t[0]
                      else "k_step_shell<float, 0, true, false>" for t in tiles)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved_tflops, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved_tflops / alu_peak, "traffic": recorded_traffic(nodes_b),
                "peak_source": "FP32 FMA issue: %d SMs (queried) x 128 lanes x 2 x 2070 MHz (recipe unit counts)"
                               % sm_count,
                "flops_per_node": flops_per_node, "nodes_per_launch": nodes_b,
                "share_of_step": shell_ms / step_ms if step_ms > 0 else None,
                "hbm": {"achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": hbm_achieved / peaks["hbm_gbs"], "peak_source": peak_kind,
                        "bytes_per_node": BYTES_PER_NODE["f32"]}}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "pores": len(pores), "nodes": nodes_b,
                       "time_steps_per_step": SUB,
                       "step": "%d time steps of every pore (CUDA-graph replays) + the FP64 flux residual of "
                               "every pore" % SUB,
                       "storage": "f32 deviation from the local rest state, FP64 reductions",
                       "l2": "no flush: populations 2 x %.0f MB exceed the 129 MB L2" % (nodes_b * 76 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "shell_kernel": {"tiles": tiles, "chosen_by": "built-in tile rule",
                                        "tma_tile_pores": tma_pores},
                       "sm_count": sm_count},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "path": "per step: wdlb_batch_add of the 64 pores from pinned host n, u; wdlb_batch_step(%d); "
                            "wdlb_moments of every pore into pinned host buffers; wdlb_batch_remove. Two batches "
                            "on their own streams alternate: the next step's admission overlaps the current "
                            "step's time steps (fill and drain timed)" % SUB,
                    "serial": {"value": e2e_vals[False], "unit": UNIT,
                               "form": "one batch: admission, time steps and read-back one after another"}},
            "clocks": clocks, "gpu_launches": int(gpu_launches),
            "kernels_ms": {"moments": kms[0], "smeared_density": kms[1], "shell_collide_stream": kms[2],
                           "source": "a second pass of the same batch launched phase by phase with CUDA events "
                                     "around each launch (%.2f ms per bench step, against %.2f ms for the graph "
                                     "replays timed for value)" % (instrumented_ms, elapsed_ms / args.steps)},
            "batched_persistent": persistent_leg, "batched_dw_collision": dw_leg,
            "paths": paths, "serve": serve, "pore_viscosity_sweep": sweep}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    global SUB, SIGMA, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--sigma", type=float, default=SIGMA,
                    help="hard-sphere diameter of the main box (lattice units); the workload is quoted at 4")
    ap.add_argument("--shell-rule", default="full", choices=["full", "compact"],
                    help="contact-shell quadrature of the main timed workload")
    ap.add_argument("--only-device", action="store_true",
                    help="time only the device-resident loop (for profiling); no e2e, baseline or other paths")
    ap.add_argument("--sub", type=int, default=SUB, help="lattice time steps per benchmark step")
    ap.add_argument("--workload", default="batch64", choices=["batch64", "bulk128"],
                    help="with --only-device: the 64-pore batch (default) or the 128^3 bulk box")
    ap.add_argument("--interactions", type=int, default=1, choices=[0, 1],
                    help="with --workload bulk128: 0 skips the shell sums (profiling the per-node work alone)")
    ap.add_argument("--tile", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="tile shape of the tiled shell kernel (-1: autotuner)")
    ap.add_argument("--collision", default="fp32", choices=["fp32", "dw"],
                    help="with --only-device: the collision arithmetic of the 64-pore batch (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    SUB = args.sub
    if args.sigma != SIGMA:
        SIGMA = args.sigma
        WORKLOAD = WORKLOAD.replace("sigma=4 lattice units", "sigma=%g lattice units" % SIGMA)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
