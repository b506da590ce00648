#!/usr/bin/env python
"""Benchmark of the PFLBM hot path on GB300: MLUPS and fraction of HBM peak.

One benchmark step = one segment of S lattice time steps of the workload (the
fused stream-collide of h and g with the phi stencil, one launch per lattice
step), run through the C interface.  Default workload: the vertical drop
impact into a pool, 512 x 384 x 512 cells (100.7 M, no-slip walls on every
face, pool depth 128, drop diameter 64 starting 8 above the surface, Weber and
Froude 200, rho ratio 1000, viscosity ratio 50, xi = 5, M = 0.02), the largest
single-GPU workload, in shifted-FP16 storage with FP32 arithmetic; S = 100, so
a run of 100 benchmark steps covers its 10000 time steps.  FP32 and FP64 are
timed on the same lattice in the same run.

  value     MLUPS with the state resident in HBM (device timing, CUDA events);
  e2e       MLUPS through the public API with host buffers: pfl_init from
            pinned host phi0, u0 and p0 (H2D), S steps, pfl_fields of phi to
            the host (D2H);
  roofline  the stream-collide kernel's algorithmic bytes per launch over its
            CUDA-event duration, against the measured HBM copy bandwidth;
  cpu_baseline  the FP64 CPU oracle on the host cores (all of them, and one)
            over a bounded sample: a 128^3 sub-box of the same initial fields
            around the impact point.

--impl reference times that oracle as the reference arm on the same sample.
Under torchrun every rank runs an independent replica (the path is a single
domain per GPU).
"""
import argparse
import copy
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
sys.path.insert(0, ROOT)

METRIC = "PFLBM MLUPS & % HBM peak, mixed vs FP64 at stated error; adjoint/forward"
UNIT = "MLUPS"
L2_BYTES = 129 * 2 ** 20

PREC_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2}
PHI_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 4}


def step_kernel_bytes(prec, engine=0, qh=15, qg=27):
    """Algorithmic bytes per cell of one stream-collide launch: every h and g
    population read once and written once (qh h and qg g populations); the
    fused two-array step (engine 0) also writes phi, the in-place step
    (engine 1) reads phi for its stencil; FP16S adds the read of the h shifts
    (phi of the writing cells, 4 B) and the write and read of the g shifts
    (p* of the writing cells in FP16, 2 + 2 B)."""
    b = 2 * (qh + qg) * PREC_BYTES[prec] + PHI_BYTES[prec]
    if prec == "fp16s":
        b += PHI_BYTES[prec] + 4
    return b


GRAPH_STEPS = 32   # the library's default steps per replayed graph (fused engine)


def step_launches(S, engine):
    """Kernel launches of one pfl_step(S): the fused engine runs S // 32 graph
    replays of 32 step kernels and one step-count kernel each, the remaining
    steps one by one and, after those, one kernel that sets the device step
    count before the next replay; the in-place engine launches the step and
    its phi pass per step."""
    if engine != 0:
        return 2 * S
    return S + S // GRAPH_STEPS + (1 if S % GRAPH_STEPS else 0)


def ideal_step_bytes(prec):
    """Algorithmic bytes per cell update of the whole step: 2 (15 + 27) S + phi read + phi write."""
    return 2 * (15 + 27) * PREC_BYTES[prec] + 2 * PHI_BYTES[prec]


def workload(name):
    from paper_2206_11637_gb300 import workloads as W
    if name == "capillary_wave":
        p, phi0, u0, p0 = W.capillary_wave(200)
        return dict(p=p, phi0=phi0, u0=u0, p0=p0, S=2000, total=20000, prec="fp16s",
                    desc="standing capillary wave 200x400x1, walls in y, rho ratio 1000, nu 0.01, sigma 1e-4, xi 5, M 0.02")
    if name == "static_drop":
        p, phi0, u0, p0 = W.static_drop(32, 10.0)
        return dict(p=p, phi0=phi0, u0=u0, p0=p0, S=100, total=1000, prec="fp64",
                    desc="static drop 32^3 periodic, R 10, xi 5, rho ratio 1000, sigma 1e-4, M 0.02")
    if name == "rising_bubble":
        p, phi0, u0, p0 = W.rising_bubble()
        return dict(p=p, phi0=phi0, u0=u0, p0=p0, S=200, total=4000, prec="fp32",
                    desc="rising bubble 128x384x128, walls, D 32, Eo 10, Mo 1e-3, xi 4, M 0.02")
    if name == "drop_impact_256":
        # the same impact at half the linear size (12.6 M cells): profiling case
        p, phi0, u0, p0 = W.drop_impact(256, 192, 256, D=32.0, depth=64.0, gap=4.0)
        return dict(p=p, phi0=phi0, u0=u0, p0=p0, S=100, total=5000, prec="fp16s",
                    crop=(96, 160, 52, 116, 96, 160),
                    desc="drop impact 256x192x256 (12.6 M cells), walls, pool depth 64, D 32 at 4 above the "
                         "surface, We 200, Fr 200, rho ratio 1000, mu ratio 50, xi 5, M 0.02")
    if name == "drop_impact":
        p, phi0, u0, p0 = W.drop_impact()
        # the CPU sample: 128^3 cells around the impact point (pool surface at
        # y = 128, drop centre at y = 168)
        return dict(p=p, phi0=phi0, u0=u0, p0=p0, S=100, total=10000, prec="fp16s",
                    crop=(192, 320, 104, 232, 192, 320),
                    desc="drop impact 512x384x512 (100.7 M cells), walls, pool depth 128, D 64 at 8 above the "
                         "surface, We 200, Fr 200, rho ratio 1000, mu ratio 50, xi 5, M 0.02")
    raise SystemExit("unknown workload " + name)


def kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "lattice.cuh", "step.cuh"):
        with open(os.path.join(ROOT, "paper_2206_11637_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per launch of the stream-collide kernel from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by workload, precision
# and the hash of the kernel sources they were taken on.  A capture of another
# kernel version does not apply.
NCU_TRAFFIC = {
    # k_step_zm<2, 15, 0, 0> (FP16S) captured on the half-size impact (256x192x256,
    # 12.58 M cells): 1.1640 GB read + 1.0975 GB written = 179.7 B/cell; the
    # launch's traffic grows with the cells it updates, so a full 100.7 M-cell
    # launch moves 179.7 x 100.66 M = 18.09 GB
    # (profiles/k_step_zm_drop_impact_256x192x256.md)
    ("drop_impact", "fp16s", "8f1ed78088adb18e"): 1.8092e10,
    # k_step_zm<1, 15, 0, 0> (FP32) on the same case: 2.2597 + 2.1340 GB = 349.2 B/cell
    ("drop_impact", "fp32", "8f1ed78088adb18e"): 3.5149e10,
}

# Warp instructions per launch of the same kernels (smsp__inst_executed.sum of
# the same captures, scaled by cells the same way), for the instruction-issue
# side of the roofline: launches that issue more than they move (FP16S) are
# bound there.
NCU_INST = {
    ("drop_impact", "fp16s", "8f1ed78088adb18e"): 5.3313e9,    # 52.96 per cell
    ("drop_impact", "fp32", "8f1ed78088adb18e"): 4.3670e9,     # 43.38 per cell
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock and throttle sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != device_index:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if parts[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def ranks_max(dist, x, device=None):
    """Max of x over all ranks of the process group (x itself without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n, rank, world):
    """The units rank takes of n independent units: rank, rank + world, ...
    (the ranks' shards partition range(n); no unit is shared)."""
    return list(range(rank, n, world))


def mlups(cells, steps, seconds):
    return cells * steps / seconds / 1e6


def oracle_sample(wl):
    """(params, phi0, u0, p0, text) of the CPU sample of a workload: the whole
    lattice, or for the drop impact a sub-box of the same initial fields (the
    oracle's 700 bytes per cell would need 70 GB of host memory for the full
    lattice); walls close the sub-box on every face."""
    p = wl["p"]
    if "crop" not in wl:
        return p, wl["phi0"], wl["u0"], wl["p0"], "the full %dx%dx%d lattice" % (p.nx, p.ny, p.nz)
    x0, x1, y0, y1, z0, z1 = wl["crop"]
    q = copy.copy(p)
    q.nx, q.ny, q.nz = x1 - x0, y1 - y0, z1 - z0
    q.bc = (1,) * 6
    sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
    phi0 = wl["phi0"][sl].copy()
    u0 = None if wl["u0"] is None else wl["u0"][(slice(None),) + sl].copy()
    p0 = None if wl["p0"] is None else wl["p0"][sl].copy()
    return q, phi0, u0, p0, ("a %dx%dx%d sub-box (x %d..%d, y %d..%d, z %d..%d) of the %dx%dx%d lattice's initial "
                             "fields, walls on its faces" % (q.nx, q.ny, q.nz, x0, x1, y0, y1, z0, z1, p.nx, p.ny, p.nz))


def cpu_oracle_rate(wl, budget_s=10.0):
    """FP64 oracle MLUPS on the host cores over a bounded sample of the
    workload, on all cores and on one core."""
    import oracle
    oracle.build_oracle()
    q, phi0, u0, p0, text = oracle_sample(wl)
    o = oracle.from_params(q, phi0, u0, p0)
    res = {}
    for threads in (os.cpu_count() or 1, 1):
        o.step(1, threads)                      # warm-up (thread pool, caches)
        t0 = time.perf_counter()
        o.step(1, threads)
        per = time.perf_counter() - t0
        n = max(1, min(2000, int(budget_s / max(per, 1e-9))))
        t0 = time.perf_counter()
        o.step(n, threads)
        dt = time.perf_counter() - t0
        res[threads] = (mlups(q.cells, n, dt), n, dt)
    allc = os.cpu_count() or 1
    v, n, dt = res[allc]
    v1, n1, dt1 = res[1]
    return dict(value=v, unit=UNIT, cores=allc, kind="oracle",
                sample="%d time steps of %s (FP64, %d threads, %.1f s)" % (n, text, allc, dt),
                single_core={"value": v1, "unit": UNIT, "cores": 1,
                             "sample": "%d time steps of the same sample (FP64, 1 thread, %.1f s)" % (n1, dt1)})


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    p, phi0, u0, p0, text = oracle_sample(wl)
    threads = os.cpu_count() or 1
    o = oracle.from_params(p, phi0, u0, p0)
    o.step(1, threads)
    t0 = time.perf_counter()
    o.step(1, threads)
    per = time.perf_counter() - t0
    # one benchmark step = a bounded sample of lattice steps (about 3 s)
    n_per = max(1, min(wl["S"], int(3.0 / max(per, 1e-9))))
    for _ in range(args.warmup):
        o.step(n_per, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(n_per, threads)
    dt = time.perf_counter() - t0
    v = mlups(p.cells, n_per * args.steps, dt)
    sample = "%d lattice steps of %s per benchmark step (FP64 oracle, %d threads)" % (n_per, text, threads)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "cells": p.cells,
                       "lattice_steps_per_step": n_per, "sample": text},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Config 4: 512 seeded instances (drops n^3, n in 24..96; waves nx x
    2nx, nx in 64..256) with their own M, xi, sigma, advanced together in FP32
    by the batched persistent launches of the fused step (CUDA graph, tuned
    shapes), S = 200 lattice steps per benchmark step (10 steps: the config's
    2000).  value = aggregate MLUPS; per-instance error against the FP64 CPU
    oracle after the same number of steps for a 16-instance subset (the 8
    smallest drops and the 8 smallest waves of this rank's shard).  Under
    torchrun the instances are sharded over the ranks (rank r takes r, r + N,
    ...), with no collective on the data path: value = all instances' cell
    updates over the slowest rank's time, "scaling" strong (the total work is
    fixed)."""
    import numpy as np
    import torch
    from paper_2206_11637_gb300 import workloads as W
    from paper_2206_11637_gb300 import build as B
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        B.build_library()
    if dist:
        dist.barrier()
    from paper_2206_11637_gb300.batch import Batch
    every = W.batched_sweep(512)
    mine = shard(len(every), rank, ws)
    inst = [every[i] for i in mine]
    cells = sum(p.cells for p, _, _, _ in every)
    t0 = time.perf_counter()
    b = Batch(inst, precision="fp32", tune=True, device=dev)
    t_init = time.perf_counter() - t0
    S = args.lattice_steps or 200
    for _ in range(args.warmup):
        b.step(S)
    torch.cuda.synchronize()
    clk = Clocks()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        b.step(S)
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop(local)
    ms = ranks_max(dist, e0.elapsed_time(e1), dev)
    out, nf, _ = b.diag(check=False)
    threads, grid, ntiles = b.shapes()
    # error of 16 instances against the FP64 oracle after the same number of steps
    n_done = b.time
    errs = []
    if not args.no_compare:
        import oracle
        oracle.build_oracle()
        drops = sorted([j for j in range(len(inst)) if inst[j][0].nz > 1], key=lambda j: inst[j][0].cells)[:8]
        waves = sorted([j for j in range(len(inst)) if inst[j][0].nz == 1], key=lambda j: inst[j][0].cells)[:8]
        for j in drops + waves:
            p, phi0, u0, p0 = inst[j]
            o = oracle.from_params(p, phi0, u0, p0)
            o.step(n_done, 0)
            ophi, _, _, ou = o.fields()
            phi, _, _, u = b.fields(j)
            umax = max(np.abs(ou).max(), 1e-300)
            errs.append({"instance": mine[j], "cells": p.cells, "nonfinite": int(nf[j]),
                         "phi_max_abs": float(np.abs(phi - ophi).max()),
                         "u_max_over_umax": float(np.abs(u - ou).max() / umax)})
            del o
    v = mlups(cells, S * args.steps, ms / 1e3)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, _ = peaks()
    bpc = 2 * 42 * 4 + 4    # fused FP32 step: populations read and written, phi written
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_sweep", "instances": len(every), "cells": cells,
                       "parallelism": "instances sharded over %d ranks" % ws if ws > 1 else "1 GPU",
                       "lattice_steps_per_step": S, "precision": "fp32",
                       "l2": "working set larger than L2"},
            "gpu_launches": (2 * S + 2 * S // 16) * args.steps, "clocks": clocks,
            "roofline": {"bound": "hbm", "achieved": v * 1e6 * bpc / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": v * 1e6 * bpc / 1e9 / peak, "traffic": None, "bytes_per_cell": bpc,
                         "kernel": "k_batch_zm (fused two-array step over the work list)"},
            "batch": {"init_s": t_init, "shapes": {"threads": threads.tolist(), "grid": grid.tolist(),
                                                    "tiles": ntiles.tolist()},
                      "lattice_steps_total": n_done,
                      "unstable_instances": int((nf > 0).sum()),
                      "error_vs_fp64_oracle_16": errs}}
    print(json.dumps(line), flush=True)


def adjoint_leg(dev, barrier, n=4000, window=1000, ny=384):
    """Adjoint over forward on the 128 x 384 x 128 rising bubble (FP32, walls,
    D 32, Eo 10, Mo 1e-3, xi 4, M 0.02): J = mean rise velocity over the last
    `window` of n = 4000 steps, gradient with respect to (M, xi, sigma),
    sqrt(n) checkpoints.  The ratio counts everything the adjoint call adds to
    the forward run it contains: (t_adjoint - t_forward) / t_forward.  ny < 384
    runs the same bubble in a shorter box (a profiling case)."""
    from paper_2206_11637_gb300 import objectives as O
    from paper_2206_11637_gb300 import workloads as W
    from paper_2206_11637_gb300.pflbm import Simulation
    p, phi0, u0, p0 = W.rising_bubble() if ny == 384 else W.rising_bubble(128, ny, 128)
    window = min(window, n)
    obs = O.rise_velocity_weights(p, phi0, n - window, n)
    fw = Simulation(p, phi0, u0, p0, precision="fp32", device=dev)
    fw.step(10)
    barrier()
    t0 = time.perf_counter()
    fw.step(n)
    barrier()
    t_fw = time.perf_counter() - t0
    del fw
    ad = Simulation(p, phi0, u0, p0, precision="fp32", device=dev)
    ad.adjoint(20, [(20, obs[1][1])])         # warm-up (kernels, workspace)
    ad = Simulation(p, phi0, u0, p0, precision="fp32", device=dev)
    barrier()
    t0 = time.perf_counter()
    J, g = ad.adjoint(n, obs)
    barrier()
    t_ad = time.perf_counter() - t0
    ws_gb = ad.lib.pfl_adjoint_workspace_bytes(ad.ctx, n) / 1e9
    del ad
    return {"workload": "rising_bubble 128x%dx128" % ny, "precision": "fp32", "lattice_steps": n,
            "objective": "mean rise velocity over steps %d..%d" % (n - window, n),
            "forward_ms": t_fw * 1e3, "adjoint_ms_incl_forward_and_recompute": t_ad * 1e3,
            "adjoint_over_forward": (t_ad - t_fw) / t_fw, "workspace_gb": ws_gb,
            "J": J, "grad_M_xi_sigma": [float(v) for v in g],
            "fd_check": adjoint_fd_check(dev, p, phi0, u0, p0, 2000) if n >= 2000 and ny == 384 else None}


def adjoint_fd_check(dev, p, phi0, u0, p0, n, rel=1e-2):
    """The adjoint gradient of the same bubble and objective over n steps (J
    over the last quarter) against central differences of forward FP32 runs
    with relative step rel.  Over 4000 steps J is no longer smooth in the
    parameters (finite differences do not converge as the step shrinks), so the
    check runs at a horizon where it is."""
    import copy
    import torch
    from paper_2206_11637_gb300 import objectives as O
    from paper_2206_11637_gb300.pflbm import Simulation
    obs = O.rise_velocity_weights(p, phi0, n - n // 4, n)
    wd = [(t, torch.from_numpy(w).to(dev)) for t, w in obs]

    def forward_J(q):
        s = Simulation(q, phi0, u0, p0, precision="fp32", device=dev)
        J = 0.0
        for t, w in sorted(wd, key=lambda a: a[0]):
            s.step(t - s.time)
            f = {"phi": torch.empty(s.N, dtype=torch.float64, device=dev)}
            s.fields(f)
            J += float(torch.dot(w, f["phi"]).item())
        del s
        torch.cuda.empty_cache()
        return J

    s = Simulation(p, phi0, u0, p0, precision="fp32", device=dev)
    _, g = s.adjoint(n, obs)
    del s
    torch.cuda.empty_cache()
    fd = []
    for name in ("mobility", "xi", "sigma"):
        v = getattr(p, name)
        pp, pm = copy.copy(p), copy.copy(p)
        setattr(pp, name, v * (1 + rel))
        setattr(pm, name, v * (1 - rel))
        fd.append((forward_J(pp) - forward_J(pm)) / (2 * rel * v))
    return {"lattice_steps": n, "objective": "mean rise velocity over steps %d..%d" % (n - n // 4, n),
            "relative_step": rel, "adjoint": [float(v) for v in g], "central_differences": fd,
            "rel_err": [abs(float(a) - b) / abs(b) for a, b in zip(g, fd)]}


# (workload, precision, lattice steps timed) of the per-config table
CONFIG_LEGS = [("static_drop", "fp64", 1000),
               ("capillary_wave", "fp64", 1000), ("capillary_wave", "fp32", 2000),
               ("capillary_wave", "fp16s", 2000),
               ("rising_bubble", "fp64", 20), ("rising_bubble", "fp32", 200), ("rising_bubble", "fp16s", 200),
               # the paper's own phase-field lattice (D3Q27 h)
               ("rising_bubble@d3q27", "fp32", 200), ("rising_bubble@d3q27", "fp16s", 200),
               # the paper's 2-D lattices (D2Q9 h and g) on the quasi-2-D wave
               ("capillary_wave@d2q9", "fp64", 1000), ("capillary_wave@d2q9", "fp32", 2000),
               ("capillary_wave@d2q9", "fp16s", 2000)]


def config_table(dev, barrier):
    """MLUPS and fraction of the HBM peak of every single-lattice workload and
    precision (CUDA events around S steps after three warm-up steps; the
    fraction counts the fused step's algorithmic bytes per cell), plus the
    batched sweep's aggregate."""
    import torch
    from paper_2206_11637_gb300.pflbm import Simulation
    peak, _ = peaks()
    rows = []
    cache = {}
    for name, prec, S in CONFIG_LEGS:
        base, _, lat = name.partition("@")
        if base not in cache:
            cache.clear()
            cache[base] = workload(base)
        wl = cache[base]
        p = copy.copy(wl["p"])
        qh = {"d3q27": 27, "d2q9": 9}.get(lat, 15)
        qg = 9 if qh == 9 else 27
        p.h_lattice = qh
        sim = Simulation(p, wl["phi0"], wl["u0"], wl["p0"], precision=prec, device=dev)
        sim.step(3)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.step(S)
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1)
        _, nf = sim.diag(check=False)
        del sim
        r = mlups(p.cells, S, ms / 1e3)
        bpc = step_kernel_bytes(prec, 0, qh, qg)
        work = p.cells * (2 * (qh + qg) * PREC_BYTES[prec] + 2 * PHI_BYTES[prec])
        rows.append({"workload": name, "cells": p.cells, "precision": prec, "lattice_steps": S, "mlups": r,
                     "bytes_per_cell": bpc, "hbm_frac": r * 1e6 * bpc / 1e9 / peak,
                     "l2_resident": work < L2_BYTES, "nonfinite_cells": nf})
    cache.clear()
    torch.cuda.empty_cache()
    # batched sweep: 512 instances in one persistent launch per class, graph replay
    from paper_2206_11637_gb300 import workloads as W
    from paper_2206_11637_gb300.batch import Batch
    inst = W.batched_sweep(512)
    cells = sum(q.cells for q, _, _, _ in inst)
    b = Batch(inst, precision="fp32", tune=True, device=dev)
    b.step(16)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(96)
    e1.record()
    barrier()
    r = mlups(cells, 96, e0.elapsed_time(e1) / 1e3)
    bpc = 2 * 42 * 4 + 4     # fused step: populations read and written, phi written
    rows.append({"workload": "batched_sweep", "instances": len(inst), "cells": cells, "precision": "fp32",
                 "lattice_steps": 96, "mlups": r, "bytes_per_cell": bpc, "hbm_frac": r * 1e6 * bpc / 1e9 / peak})
    del b
    torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="drop_impact",
                    choices=["capillary_wave", "static_drop", "rising_bubble", "drop_impact", "drop_impact_256",
                             "batched_sweep"])
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32", "fp16s"])
    ap.add_argument("--lattice-steps", type=int, default=None, help="lattice steps per benchmark step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precisions")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="N",
                    help="run only the adjoint leg over N steps and print its JSON (profiling)")
    ap.add_argument("--adjoint-ny", type=int, default=384, metavar="NY",
                    help="height of the adjoint leg's bubble box (384: the config; less for profiling)")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 1],
                    help="0: fused two-array step (default), 1: in-place AA step + phi pass")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.adjoint_only:
        import torch
        from paper_2206_11637_gb300 import build as B
        B.build_library()
        torch.cuda.set_device(0)
        r = adjoint_leg(torch.device("cuda", 0), torch.cuda.synchronize, args.adjoint_only, ny=args.adjoint_ny)
        print(json.dumps(r), flush=True)
        return
    if args.workload == "batched_sweep":
        return run_batched(args)
    wl = workload(args.workload)
    wl["p"].engine = args.engine
    if args.lattice_steps:
        wl["S"] = args.lattice_steps
    if args.impl == "reference":
        return run_reference(args, wl)

    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2206_11637_gb300 import build as B
    if rank == 0 or ws == 1:
        B.build_library()
    if dist:
        dist.barrier()
    from paper_2206_11637_gb300.pflbm import Simulation

    p = wl["p"]
    N = p.cells
    S = wl["S"]
    prec = args.precision or wl["prec"]
    work_bytes = N * (2 * 42 * PREC_BYTES[prec] // 2 + 2 * PHI_BYTES[prec])
    flush = work_bytes < 4 * L2_BYTES
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if flush else None
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_device(precision, K, Wm, S=S):
        sim = Simulation(p, wl["phi0"], wl["u0"], wl["p0"], precision=precision, device=dev)
        for _ in range(Wm):
            sim.step(S)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        clk = Clocks()
        if precision == prec:
            clk.start()
        t0 = time.perf_counter()
        for k in range(K):
            if flush:
                flush_buf.fill_(float(k))
            evs[k][0].record(stream)
            sim.step(S)
            evs[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
        clocks = clk.stop(dev.index or 0) if precision == prec else None
        ms = sum(a.elapsed_time(b) for a, b in evs)
        out, nf = sim.diag(check=False)
        return sim, ms, wall, clocks, nf

    K, Wm = args.steps, args.warmup
    sim, ms, wall, clocks, nf = timed_device(prec, K, Wm)
    ms = ranks_max(dist, ms, dev)
    value = mlups(N, S * K, ms / 1e3) * ws

    # roofline of the stream-collide kernel.  With the fused engine the timed
    # region launches that kernel alone, once per lattice step, so its average
    # launch duration is the region's device time over the launch count.  The
    # in-place engine also runs the phi pass: its share comes from CUDA events
    # around each of the two launches of a few extra steps.
    n_rt = min(S, 400)
    if args.engine == 0:
        kms, pms = ms, 0.0
        avg_s = ms / (S * K) / 1e3
    else:
        kms, pms = sim.kernel_times(n_rt)
        avg_s = ms / (S * K) / 1e3 * kms / (kms + pms)
    peak, peak_kind = peaks()
    achieved = N * step_kernel_bytes(prec, args.engine) / avg_s / 1e9
    traffic = NCU_TRAFFIC.get((args.workload, prec, kernel_hash()))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": "k_step_zm (fused two-array step)" if args.engine == 0 else "k_step_mrt (in-place step)",
                "bytes_per_cell": step_kernel_bytes(prec, args.engine), "peak_source": peak_kind,
                "kernel_share": kms / (kms + pms),
                "whole_step_ideal_frac": mlups(N, S * K, ms / 1e3) * 1e6 * ideal_step_bytes(prec) / 1e9 / peak,
                "working_set_bytes": work_bytes, "l2_resident": work_bytes < L2_BYTES}
    inst = NCU_INST.get((args.workload, prec, kernel_hash()))
    if inst is not None and args.engine == 0:
        # issue side: 4 warp instructions per SM per clock at the maximum SM clock
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        ipeak = sms * 4 * mhz * 1e6
        roofline["issue"] = {"achieved": inst / avg_s, "peak": ipeak, "unit": "warp instructions/s",
                             "frac": inst / avg_s / ipeak, "inst_per_launch": inst, "sms": sms, "sm_mhz": mhz,
                             "source": "smsp__inst_executed.sum of one ncu capture of this kernel version"}
    del sim

    # e2e through the public API with host buffers: every input of the
    # workload (phi0, u0, p0) from pinned host memory, phi back to the host
    def pinned(a):
        if a is None:
            return None
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).pin_memory()

    ins = [pinned(wl["phi0"]), pinned(wl["u0"]), pinned(wl["p0"])]
    h2d = sum(t.numel() * 8 for t in ins if t is not None)
    phi_out = torch.empty(N, dtype=torch.float64).pin_memory()
    from paper_2206_11637_gb300 import _lib as L
    import ctypes

    def e2e_once():
        s = Simulation(p, ins[0], ins[1], ins[2], precision=prec, device=dev)
        s.step(S)
        L.check(s.lib.pfl_fields(s.ctx, ctypes.c_void_p(phi_out.data_ptr()), None, None, None))
        s.close()

    for _ in range(2):
        e2e_once()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_once()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": mlups(N, S * K, e2e_s) * ws, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": N * 8}
    del ins, phi_out
    torch.cuda.empty_cache()

    # the other precisions (FP64 over fewer lattice steps per benchmark step:
    # it runs ~15x slower) and the error of FP32 and FP16S against FP64 after
    # 1000 lattice steps (max |dphi| and max |du| / max |u|), on the device
    compare = {}
    leg_errors = {}

    def leg(name, fn):
        """Run an auxiliary leg after the headline measurement; a failure is
        recorded in the line (leg_errors) instead of losing the line."""
        try:
            return fn()
        except Exception as e:  # noqa: BLE001 -- reported, not hidden
            leg_errors[name] = "%s: %s" % (type(e).__name__, e)
            torch.cuda.empty_cache()
            return None

    def compare_leg():
        for other in ("fp64", "fp32", "fp16s"):
            if other == prec:
                continue
            S_o = max(4, S // 5) if other == "fp64" else S
            s2, ms2, _, _, _ = timed_device(other, max(2, K // 3), 3, S_o)
            compare[other + "_mlups"] = mlups(N, S_o * max(2, K // 3), ms2 / 1e3)
            del s2
            torch.cuda.empty_cache()
        compare["speedup_vs_fp64"] = value / ws / compare["fp64_mlups"] if "fp64_mlups" in compare else None
        n_acc = min(wl["total"], 1000)
        marks = [m for m in (100, 250, 500) if m < n_acc] + [n_acc]

        def dev_fields(precision):
            """phi and u (FP32 copies, on the device) at the marks."""
            s3 = Simulation(p, wl["phi0"], wl["u0"], wl["p0"], precision=precision, device=dev)
            out = []
            for m in marks:
                s3.step(m - s3.time)
                f = {"phi": torch.empty(N, dtype=torch.float64, device=dev),
                     "u": torch.empty(3 * N, dtype=torch.float64, device=dev)}
                s3.fields(f)
                out.append({"phi": f["phi"].float(), "u": f["u"].float()})
                del f
            del s3
            torch.cuda.empty_cache()
            return out

        f64 = dev_fields("fp64")
        errs = {"lattice_steps": n_acc, "marks": marks,
                "u_max": [max(r["u"].abs().max().item(), 1e-300) for r in f64],
                "measure": "max over cells (and components) of |x - x_fp64|, u divided by max |u_fp64|; rms the "
                           "root mean square over cells"}
        for other in ("fp32", "fp16s"):
            ft = dev_fields(other)
            e = {"phi_max_abs": [], "phi_rms": [], "u_max_over_umax": [], "u_rms_over_umax": []}
            for a, r, um in zip(ft, f64, errs["u_max"]):
                dphi = (a["phi"] - r["phi"]).abs()
                du = (a["u"] - r["u"]).abs()
                e["phi_max_abs"].append(dphi.max().item())
                e["phi_rms"].append(dphi.pow(2).mean().sqrt().item())
                e["u_max_over_umax"].append(du.max().item() / um)
                e["u_rms_over_umax"].append(du.pow(2).mean().sqrt().item() / um)
            errs[other] = e
            del ft
        last = -1
        compare["error_vs_fp64"] = dict(errs, phi_max_abs=errs[prec]["phi_max_abs"][last] if prec != "fp64" else 0.0,
                                        u_max_over_umax=errs[prec]["u_max_over_umax"][last] if prec != "fp64" else 0.0)
        del f64
        torch.cuda.empty_cache()

    adj = None
    configs = None
    if not args.no_compare and rank == 0:
        leg("compare", compare_leg)
        adj = leg("adjoint", lambda: adjoint_leg(dev, barrier))
        configs = leg("configs", lambda: config_table(dev, barrier))

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = leg("cpu_baseline", lambda: cpu_oracle_rate(wl))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f16 storage / f32 arithmetic" if prec == "fp16s" else ("f32" if prec == "fp32" else "f64"),
                "data": "synthetic",
                "config": {"workload": args.workload, "description": wl["desc"], "precision": prec,
                           "cells": N, "lattice_steps_per_step": S, "parallelism": "replicas" if ws > 1 else "1 GPU",
                           "l2": ("L2 flushed before each timed benchmark step of %d lattice steps" % S) if flush else "working set larger than L2"},
                "e2e": e2e, "gpu_launches": step_launches(S, args.engine) * K, "clocks": clocks, "roofline": roofline,
                "cpu_baseline": cpu, "nonfinite_cells": nf, "wall_s": wall, "adjoint": adj,
                "configs": configs}
        if leg_errors:
            line["leg_errors"] = leg_errors
        line.update(compare)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
