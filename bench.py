#!/usr/bin/env python3
"""Benchmark of the geometric VoF advection step (one JSON line on rank 0).

Workload (default): 128^3 hexahedral mesh on [0,1]^3 with interior points
jittered by +-0.2h (seed 1302), sphere R=0.15 at (0.35,0.35,0.35), deformation
field (T=3), Courant number 0.5.  A step is one full vof_advect call (band
classification, reconstruction, point velocities, flux correction, phase
fluxes, update and bounding) with the step's flux F and cell velocity U_c
already resident in HBM.  Metric: internal face fluxes with final phase volume
per second (millions), whole job.

--workload batch: the batched form -- independent cases of uneven size (half
hexahedral boxes n^3, n in [16, 64], half Kuhn-split lattices n in [16, 48],
each with a random sphere or plane under a solid-body rotation at Courant
0.3-0.8; --cases, --batch-scale shrinks the size ranges) advanced as one mesh,
one CUDA-graph launch per step, phase-flux launch shape from the autotuner.

--impl reference times the CPU oracle (test infrastructure) on the host cores
on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "geometric VoF face fluxes/s (M/s), mixed vs plain FP64 GPU, at stated L1 error"
UNIT = "M face fluxes/s"
# Algorithmic flop cost of each primitive the step kernels count (vof_work_counts;
# signed point-plane distance 6 = 3 FMA, edge intersection 10 including its
# division, tetrahedron volume 17, closed-form cut fraction 30 = three
# division-bearing edge parameters and their product):
#  - phase flux, FP32 in the mixed form and FP64 in the plain one: six
#    distances per prism-plane set, four per piece-plane test, the rest as named
PF_FLOPS = {"prism_planes": 6 * 6, "piece_tests": 4 * 6, "edges": 10, "tet_volumes": 17, "cut_fractions": 30,
            "plane_shifts": 6}
#  - positioning: one fill evaluation of a cell tetrahedron (sorted projections,
#    closed-form cut fraction and its derivative) 30, FP64 or FP32 as counted
FILL_FLOPS = 30
#  - correction (FP64): the cubic's coefficients from one swept face triangle
#    (E1, E2, the summed stream vector and four 3x3 determinants) 110, one cubic
#    evaluation with its scale and Newton step 20
CTRI_FLOPS, CEVAL_FLOPS = 110, 20
# algorithmic HBM bytes per internal face and step (flux 8, owner/neighbour 8,
# face point indices 20, alpha r/w and volume 8, point data 28)
BYTES_PER_FACE = 72.0

# DRAM bytes per launch of the mixed phase-flux kernel: dram__bytes_read.sum +
# dram__bytes_write.sum, mean of the two timed launches of one ncu capture of
# the default launch shape (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,
# gpu__time_duration.sum -k regex:k_phase_flux_mixed -s 3 -c 3 python bench.py
# --steps 2 --warmup 3 --no-tune --no-cpu-baseline --fp64-steps 0 --full-run 0);
# valid while the kernel's sources hash to the captured digest, else null.
TRAFFIC = {
    ("deform3d", 128, "mixed"): {"bytes": 68.08e6, "sources_sha256": "a46f217f59e4de731bd9a6d310010b01930eabe90b9d14362bd5b68a8c8addaf"},
}
TRAFFIC_SOURCES = ["paper_1305_3417_gb300/csrc/vof_phase_flux.cu", "paper_1305_3417_gb300/csrc/vof_device.cuh"]


def captured_traffic(workload, n, precision):
    t = TRAFFIC.get((workload, n, precision))
    if t is None:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return t["bytes"] if h.hexdigest() == t["sources_sha256"] else None


def work_flops(work, fp64_phase_flux):
    """(FP32 flops, FP64 flops, phase-flux flops) of counted work."""
    pf = sum(work[k] * v for k, v in PF_FLOPS.items())
    f32 = work["fill32"] * FILL_FLOPS
    f64 = work["fill64"] * FILL_FLOPS + work["cubic_triangles"] * CTRI_FLOPS + work["cubic_evals"] * CEVAL_FLOPS
    if fp64_phase_flux:
        f64 += pf
    else:
        f32 += pf
    return f32, f64, pf


def counted_work(ctx, alpha, steps):
    """The algorithmic work of the given steps (list of (U, F, dt)), counted by
    the instrumented kernels from the state alpha (a copy is advanced; the
    timed steps ran the uninstrumented kernels from the same state).  Per step."""
    import torch
    from paper_1305_3417_gb300 import vof
    a = alpha.clone()
    st = torch.zeros(vof.S_LEN, dtype=torch.float64, device=alpha.device)
    vof.vof_work_counts(ctx.h, reset=True)
    vof.vof_count_work(ctx.h, True)
    for U, F, dt in steps:
        ctx.advect(a, U, F, dt, st)
    torch.cuda.synchronize()
    vof.vof_count_work(ctx.h, False)
    w = vof.vof_work_counts(ctx.h, reset=True)
    return {k: v / max(len(steps), 1) for k, v in w.items()}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, idx):
        self.idx = idx
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_link_gbps(stream, host):
    """Copy bandwidth between pinned host memory and the device on this machine
    (GB/s, three timed copies each way of the given pinned tensor): the host
    link bounds the end-to-end number, whose copies are in its timed region."""
    import torch
    dev = torch.empty_like(host, device="cuda")
    out = {}
    for name, dst, src in (("h2d", dev, host), ("d2h", host, dev)):
        dst.copy_(src, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = 3 * host.numel() * host.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev
    return out


def host_buffers_diag(stream, bufs, device):
    """Where the end-to-end copies' time goes: H2D rate of each pinned buffer
    copied alone (GB/s: min, median, max), whether all are pinned, and the
    GPU's NUMA node and local CPUs as the kernel reports them."""
    import torch
    rates = []
    for b in bufs:
        dst = torch.empty_like(b, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dst.copy_(b, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        rates.append(b.numel() * b.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        del dst
    out = {"h2d_GBps_per_buffer": {"min": float(np.min(rates)), "median": float(np.median(rates)),
                                   "max": float(np.max(rates)), "buffers": len(rates)},
           "pinned": bool(all(b.is_pinned() for b in bufs))}
    try:
        bus = torch.cuda.get_device_properties(device).pci_bus_id.lower()
        base = f"/sys/bus/pci/devices/{bus}"
        with open(base + "/numa_node") as f:
            out["gpu_numa_node"] = int(f.read().strip())
        with open(base + "/local_cpulist") as f:
            out["gpu_local_cpus"] = f.read().strip()
    except Exception:
        pass
    try:
        out["process_cpus"] = len(os.sched_getaffinity(0))
    except Exception:
        pass
    return out


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    from paper_1305_3417_gb300 import inputs as I
    return I.make_workload(args.workload, n=args.n)


def cpu_model():
    """The host CPU's model name (lscpu), or the platform's processor string."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w, steps=1, warmup=0, one_thread=False):
    """The oracle as it stands, timed on the host cores on full steps of the
    same workload (after `warmup` untimed ones); with one_thread, one more step
    timed on a single thread beside it."""
    from oracle import oracle as O
    threads = O.set_threads(os.cpu_count() or 1)
    om = O.OracleMesh(w.mesh)
    a = w.alpha0.copy()
    for k in range(warmup):
        F, U, dt = w.step_inputs(k)
        a, st, s = om.advect(a, U, F, dt)
    t_total = 0.0
    for k in range(warmup, warmup + steps):
        F, U, dt = w.step_inputs(k)
        t0 = time.perf_counter()
        a, st, s = om.advect(a, U, F, dt)
        t_total += time.perf_counter() - t0
    v = steps * w.mesh.n_internal / t_total / 1e6
    one = None
    if one_thread:
        O.set_threads(1)
        F, U, dt = w.step_inputs(warmup + steps)
        t1 = time.perf_counter()
        om.advect(a, U, F, dt)
        t1 = time.perf_counter() - t1
        O.set_threads(threads)
        one = {"value": w.mesh.n_internal / t1 / 1e6, "cores": 1, "sample": f"1 full oracle step, {t1:.1f} s"}
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "one_thread": one,
            "sample": f"{steps} full oracle step(s) of the {args_workload_name(w)} workload after {warmup} "
                      f"untimed one(s) from t=0 "
                      f"({w.mesh.n_internal} internal faces each), {t_total:.1f} s"}, st


def args_workload_name(w):
    return f"{w.name} {w.mesh.shape}"


def run_reference(args, world, rank):
    if rank != 0:
        return
    w = workload(args)
    base, st = cpu_baseline(w, steps=max(1, args.steps), warmup=max(0, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": 1,
            "steps": max(1, args.steps), "warmup": max(0, args.warmup),
            "ms_per_step": w.mesh.n_internal / (base["value"] * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, w),
            "cpu_baseline": {**base, "value": base["value"]},
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(args, w):
    m = w.mesh
    if m.kind == "octree":
        desc = (f"{w.name}: octree on a {m.shape[0]}^3 base lattice split twice near the sphere (finest h = "
                f"1/{round(1 / m.h)}), 2:1 balanced ({m.n_cells} cells, {m.n_internal} internal faces), "
                f"{w.field.name} field, Co 0.5 on the finest cells")
    else:
        desc = (f"{w.name}: {m.shape[0]}x{m.shape[1]}x{m.shape[2]} {m.kind} mesh "
                f"({m.n_cells} cells, {m.n_internal} internal faces), jitter, {w.field.name} field, Co 0.5")
    return {"workload": desc,
            "n_cells": m.n_cells, "n_internal_faces": m.n_internal, "precision": args.precision,
            "learned_guess": bool(args.mlp), "skip_steps": args.skip, "dt": w.dt,
            "l2": "inputs larger than L2 (mesh, fluxes and per-step arrays > 129 MB)"}


def train_guess(device, workload="deform3d"):
    """The initial-guess network trained on seeded sphere/plane fields (volume
    fractions computed on the device) of a 96^3 jittered hexahedral mesh,
    about 10^6 interface cells over 180 fields, or for the octree workload of
    a 32^3-based two-level octree (cells like the workload's: boxes of three
    sizes with hanging points); targets from the FP64 reconstruction."""
    import torch
    from paper_1305_3417_gb300 import inputs as I, mlp, vof
    t0 = time.perf_counter()
    if workload == "octree":
        m, nf = I.octree_mesh(32, 2), 120
    else:
        m, nf = I.hex_mesh((96, 96, 96), jitter=0.2, seed=21), 180
    c64 = vof.VofContext(m, precision=vof.FP64, device=device)
    X, Y = mlp.samples(c64, m, mlp.random_fields_device(c64, m, nf, seed=22))
    net = vof.Mlp(mlp.init_params(1306), max_batch=1 << 17, device=device)
    hist = mlp.train(net, X, Y, epochs=30, batch=4096, lr=3e-3)
    torch.cuda.synchronize()
    return {"net": net, "samples": int(X.shape[0]), "loss_first": hist[0], "loss_last": hist[-1],
            "train_s": time.perf_counter() - t0}


def full_run_l1(ctx, w, dev):
    """The whole case, t = 0 to the workload's end time, on the device (inputs
    formed on the device from the spatial fields with the same time factors as
    the timed steps, the last step trimmed to land on the end time), then the L1
    shape error sum_c V_c |alpha_c(t_end) - alpha_c(0)|: the deformation and
    vortex fields reverse (cos(pi t / T)), so the exact state at t_end = T is
    the initial one.  Also the relative volume change over the run."""
    import torch
    from paper_1305_3417_gb300 import vof
    Fs = torch.from_numpy(w.F_spatial).to(dev)
    Us = torch.from_numpy(np.ascontiguousarray(w.U_spatial).reshape(-1)).to(dev)
    a0 = torch.from_numpy(w.alpha0.copy()).to(dev)
    a = a0.clone()
    st = torch.zeros(vof.S_LEN, dtype=torch.float64, device=dev)
    f = w.field
    ctx.status()
    # the step inputs of the whole case formed first (device), so that the
    # events below time the steps alone
    sched, t = [], 0.0
    while t < w.t_end - 1e-12 * w.t_end:
        dt = min(w.dt, w.t_end - t)
        sched.append((t, dt))
        t += dt
    n = len(sched)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_ms = 0.0
    t0 = time.perf_counter()
    for i0 in range(0, n, 64):
        chunk = [(Us * f.tau(t + 0.5 * dt), Fs * ((f.tau_int(t + dt) - f.tau_int(t)) / dt), dt)
                 for t, dt in sched[i0:i0 + 64]]
        e0.record(stream)
        for U, F, dt in chunk:
            ctx.advect(a, U, F, dt, st)
        e1.record(stream)
        torch.cuda.synchronize()
        gpu_ms += e0.elapsed_time(e1)
    secs = time.perf_counter() - t0
    vc = ctx.geometry()[1]
    m0 = float((vc * a0).sum())
    l1 = float((vc * (a - a0).abs()).sum())
    return {"t_end": w.t_end, "steps": n, "l1": l1, "l1_rel_to_initial_volume": l1 / m0,
            "rel_volume_change": float((vc * a).sum()) / m0 - 1.0, "alpha_min": float(a.min()),
            "alpha_max": float(a.max()), "status_bits": int(ctx.status()), "wall_s": secs, "gpu_ms": gpu_ms}


def positioning_iterations(ctx, alpha, net):
    """Mean positioning iterations per oriented interface cell, without and
    with the network, on the state alpha (vof_reconstruct)."""
    from paper_1305_3417_gb300 import vof
    out = []
    for q in (None, net):
        vof.vof_set_guess(ctx.h, q)
        _, _, fl, it = ctx.reconstruct(alpha)
        sel = (fl & 2) != 0
        out.append(float(it[sel].double().mean()))
    vof.vof_set_guess(ctx.h, net)
    return out


def make_batch(args):
    from paper_1305_3417_gb300 import inputs as I
    s = args.batch_scale
    hr = (max(4, round(16 * s)), max(4, round(64 * s)))
    tr = (max(3, round(16 * s)), max(3, round(48 * s)))
    return I.make_batch(args.cases, seed=1304, hex_range=hr, tet_range=tr, steps=50), hr, tr


def batch_config(args, b, hr, tr, tune):
    m = b.mesh
    nh = sum(c.kind == "hex" for c in b.cases)
    return {"workload": f"batch: {len(b.cases)} cases ({nh} hex n in {list(hr)}, {len(b.cases) - nh} Kuhn tet n in "
                        f"{list(tr)}), sphere or plane, solid-body rotation, Co 0.3-0.8, seed 1304 "
                        f"({m.n_cells} cells, {m.n_internal} internal faces)",
            "n_cells": m.n_cells, "n_internal_faces": m.n_internal, "precision": "mixed", "cases": len(b.cases),
            "batch_scale": args.batch_scale, "graph": True, "tuned_config": tune,
            "l2": "inputs larger than L2" if m.n_cells * 48 > 129e6 else "inputs smaller than L2 (batch scale)"}


def batch_cpu_baseline(b, ncase=4):
    """The oracle on a bounded sample: one step of each of the first ncase cases."""
    from oracle import oracle as O
    threads = O.set_threads(os.cpu_count() or 1)
    faces, t = 0, 0.0
    for i in range(min(ncase, len(b.cases))):
        om = O.OracleMesh(b.meshes[i])
        t0 = time.perf_counter()
        om.advect(b.alpha_case[i].copy(), b.U_case[i], b.F_case[i], b.cases[i].dt)
        t += time.perf_counter() - t0
        faces += b.meshes[i].n_internal
    return {"value": faces / t / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one oracle step of each of the first {min(ncase, len(b.cases))} cases "
                      f"({faces} internal faces), {t:.1f} s"}


def run_batch(args, world, rank, local):
    b, hr, tr = make_batch(args)
    m = b.mesh
    if args.impl == "reference":
        if rank == 0:
            base = batch_cpu_baseline(b, ncase=max(1, args.steps))
            line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": 1,
                    "steps": max(1, args.steps), "warmup": 0, "ms_per_step": m.n_internal / base["value"] / 1e3,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                    "data": "synthetic", "config": batch_config(args, b, hr, tr, None), "cpu_baseline": base,
                    "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        return
    import torch
    from paper_1305_3417_gb300 import build, vof
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bt = vof.VofBatch(b, precision=vof.MIXED, device=local)
    ctx = bt.context()
    U = torch.from_numpy(b.U_dt.reshape(-1).copy()).to(dev)
    F = torch.from_numpy(b.F_dt.copy()).to(dev)
    alpha = torch.from_numpy(b.alpha0.copy()).to(dev)
    tune, tune_ms = bt.tune(alpha, U, F)
    mass0 = torch.zeros(len(b.cases), dtype=torch.float64, device=dev)
    mass = torch.zeros_like(mass0)
    stats = torch.zeros(vof.S_LEN, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        bt.advect(alpha, U, F, stats, mass0)
    torch.cuda.synchronize()
    a_start = alpha.clone()  # the end-to-end steps start from the same state
    st0 = vof.vof_status(ctx)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            bt.advect(alpha, U, F, stats, mass)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_max = max_over_ranks(e0.elapsed_time(e1), world, dev)
    faces = world * args.steps * m.n_internal
    value = faces / (ms_max * 1e-3) / 1e6
    # per-case mass change over the timed steps, against the boundary flux it allows
    m0, m1 = mass0.cpu().numpy(), mass.cpu().numpy()
    S = stats.cpu().numpy()
    st1 = vof.vof_status(ctx)
    # kernel groups (direct launches, profiled; the graph holds the same
    # kernels), then the same steps' work from the instrumented kernels
    pa = alpha.clone()
    vof.vof_profile_begin(ctx, 3)
    for _ in range(3):
        vof.vof_advect(ctx, pa, U, F, 1.0, stats)
    group_ms, nprof = vof.vof_profile_end(ctx)
    launches = vof.vof_last_launch_count(ctx) * args.steps
    per_launch = {g: v / max(nprof, 1) for g, v in group_ms.items()}
    pa = alpha.clone()
    vof.vof_work_counts(ctx, reset=True)
    vof.vof_count_work(ctx, True)
    for _ in range(3):
        vof.vof_advect(ctx, pa, U, F, 1.0, stats)
    torch.cuda.synchronize()
    vof.vof_count_work(ctx, False)
    work = {k: v / 3 for k, v in vof.vof_work_counts(ctx, reset=True).items()}
    f32, f64, pf = work_flops(work, False)
    alu = vof.vof_probe_fma(local, vof.MIXED)
    achieved = pf / (per_launch["phase_flux"] * 1e-3) / 1e12
    roof = {"kernel": "k_phase_flux_mixed", "bound": "alu", "achieved": achieved, "peak": alu / 1e12,
            "unit": "TFLOP/s", "frac": achieved * 1e12 / alu, "traffic": None,
            "peak_source": "measured FP32 FMA probe (vof_probe_fma)", "group_ms_per_step": per_launch,
            "work_per_launch": work, "flops_per_launch": pf}
    # end to end through the batched call itself: every step copies alpha, U
    # and F from pinned host memory, replays the step and reads alpha back
    ha = a_start.cpu().pin_memory()
    hU, hF = U.cpu().pin_memory(), F.cpu().pin_memory()
    da, dU, dF = torch.empty_like(alpha), torch.empty_like(U), torch.empty_like(F)

    def host_step():
        da.copy_(ha, non_blocking=True)
        dU.copy_(hU, non_blocking=True)
        dF.copy_(hF, non_blocking=True)
        bt.advect(da, dU, dF, stats, mass)
        ha.copy_(da, non_blocking=True)

    host_step()  # (the graph is captured again for these buffers)
    torch.cuda.synchronize()
    ha.copy_(a_start.cpu())
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        host_step()
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e2.elapsed_time(e3), world, dev) / args.steps
    e2e = faces / (e2e_ms * args.steps * 1e-3) / 1e6
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = batch_cpu_baseline(b, ncase=args.cpu_steps * 4)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": batch_config(args, b, hr, tr, {"config": tune, "ms": tune_ms}),
                "e2e": {"value": e2e, "unit": UNIT, "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": ha.numel() * 8 + hU.numel() * 8 + hF.numel() * 8,
                        "d2h_bytes_per_step": ha.numel() * 8},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": base, "clocks": clk.summary(),
                "quality": {"rel_volume_drift_last_step": float(abs(S[1] + S[10] - S[0]) / S[0]),
                            "case_mass_min": float(m1.min()),
                            "alpha_min": float(S[4]), "alpha_max": float(S[5]),
                            "band_faces_last_step": float(S[7]), "status_bits": int(st0 | st1)}}
        print(json.dumps(line), flush=True)


def run_amr(args, world, rank, local):
    """The deformation case on a re-refined octree (Sec. 3, Alg. 2) to t = T:
    base n^3 (default 32), two levels, re-refined around the interface every
    --amr-every steps.  value: internal face fluxes per second of the device
    steps; also the whole run's wall-clock rate with the host refinement
    cycles, the remap kernel's time, the volume change across remaps and the
    L1 error at t = T against the sphere's fractions on the final mesh."""
    import torch
    from paper_1305_3417_gb300 import amr, build, vof
    from paper_1305_3417_gb300 import inputs as I
    build.build()
    torch.cuda.set_device(local)
    case = amr.AmrCase(n0=args.n or 32, levels=2, band=3.0, precision=vof.MIXED, every=args.amr_every,
                       device=local)
    stream = torch.cuda.current_stream()
    stats = torch.zeros(vof.S_LEN, dtype=torch.float64, device="cuda")
    v0 = case.volume()
    dev_ms, faces, t_remap, cells = 0.0, 0, 0.0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    worst_drift, lo, hi = 0.0, 1.0, 0.0
    wall0 = time.perf_counter()
    with Clocks(local) as clk:
        while case.t < 3.0 - 1e-12:
            if case.steps and case.steps % case.every == 0:
                r0 = time.perf_counter()
                case.remap()
                t_remap += time.perf_counter() - r0
            cells.append(case.mesh.n_cells)
            e0.record(stream)
            case.step(3.0, stats)
            e1.record(stream)
            torch.cuda.synchronize()
            dev_ms += e0.elapsed_time(e1)
            faces += case.mesh.n_internal
            s_ = stats.cpu().numpy()
            worst_drift = max(worst_drift, abs(s_[1] - s_[0]) / s_[0])
            lo, hi = min(lo, s_[4]), max(hi, s_[5])
    wall = time.perf_counter() - wall0
    ex = I.sampled_fraction(case.mesh, I.sphere_sdf(case.center, case.R))
    a = case.alpha.cpu().numpy()
    vc = case.vc.cpu().numpy()
    l1 = float((vc * np.abs(a - ex)).sum())
    if rank == 0:
        line = {"metric": METRIC, "value": faces / (dev_ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1,
                "steps": case.steps, "warmup": 0, "ms_per_step": dev_ms / case.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"octree_amr: {args.n or 32}^3 base, two levels, deformation field to t = T = 3, "
                                       f"re-refined every {case.every} steps (Sec. 3, Alg. 2)",
                           "cells_min": int(min(cells)), "cells_max": int(max(cells)), "remaps": case.remaps},
                "whole_run": {"wall_s": wall, "value_with_remaps": faces / wall / 1e6, "remap_wall_s": t_remap},
                "clocks": clk.summary(),
                "quality": {"max_rel_volume_drift": worst_drift, "alpha_min": lo, "alpha_max": hi,
                            "max_remap_volume_change": max(abs(x) for x in case.mass_change),
                            "rel_volume_change": case.volume() / v0 - 1.0, "l1_at_T": l1,
                            "l1_rel_to_volume": l1 / float((vc * ex).sum())}}
        print(json.dumps(line), flush=True)


def run_accuracy(args, world, rank, local):
    """Reconstruction accuracy (Sec. 4.1) at scale: a jittered n^3 hexahedral
    mesh (default 128) holding a ball (R = 0.27 at (0.41, 0.47, 0.52)) as its
    E_vsd routine resolves it; the reconstruction with the NAG and with the
    generalised LSQ gradient (Sec. 2.2.1), E_vsd of each, and the times of the
    LSQ gradient (every cell) and of E_vsd.  The LSQ gradient is FP64-bound:
    per neighbour the offset (3), its squared length (5), the inverse (an FP64
    division, counted 20), the weighted offset (3) and nine accumulations
    (18): 49 flop; per cell the adjugate solve, 60 flop; against the measured
    FP64 FMA rate (its 164 B per cell of HBM traffic take 0.05 ms here)."""
    import torch
    from paper_1305_3417_gb300 import build, vof
    from paper_1305_3417_gb300 import inputs as I
    build.build()
    torch.cuda.set_device(local)
    n = args.n or 128
    m = I.hex_mesh((n, n, n), jitter=0.2, seed=1302)
    ctx = vof.VofContext(m, precision=vof.FP64, device=local)
    ball, levels = (0.41, 0.47, 0.52, 0.27), 4
    vc = ctx.geometry()[1]
    vb = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    vof.vof_evsd(ctx.h, None, None, None, ball, levels, vb)
    a = torch.clamp(vb / vc, 0.0, 1.0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    g = torch.zeros(3 * m.n_cells, dtype=torch.float64, device="cuda")
    vof.vof_set_gradient(ctx.h, vof.GRAD_LSQ)
    t_lsq = timed(lambda: vof.vof_lsq_gradient(ctx.h, a, g))
    out = {}
    ev = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    pk, pk_src = peaks()
    for kind, name in ((vof.GRAD_NAG, "nag"), (vof.GRAD_LSQ, "lsq")):
        vof.vof_set_gradient(ctx.h, kind)
        nn, dd, fl, _ = ctx.reconstruct(a)
        t_ev = timed(lambda: vof.vof_evsd(ctx.h, fl, nn, dd, ball, levels, ev), reps=2)
        out[name] = {"evsd": float(ev.sum()), "evsd_rel_to_volume": float(ev.sum() / (vc * a).sum()),
                     "interface_cells": int(((fl & 1) != 0).sum()), "evsd_ms": t_ev}
    # cells sharing a point with a cell of the n^3 lattice: 3 per axis inside,
    # 2 on the boundary, less the cell itself
    nbrs = (3 * n - 2) ** 3 - n ** 3
    flops = 49.0 * nbrs + 60.0 * m.n_cells
    p64 = vof.vof_probe_fma(local, vof.FP64)
    if rank == 0:
        line = {"metric": "reconstruction error E_vsd (Sec. 4.1) and LSQ gradient throughput", "value": out["lsq"]["evsd"],
                "unit": "E_vsd volume", "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": False,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"accuracy: {n}^3 jittered hex, ball R = 0.27, {levels} levels", "n_cells": m.n_cells},
                "lsq_gradient": {"ms": t_lsq, "cells_per_s": m.n_cells / (t_lsq * 1e-3),
                                 "roofline": {"bound": "alu", "achieved": flops / (t_lsq * 1e-3) / 1e12,
                                              "peak": p64 / 1e12, "unit": "TFLOP/s",
                                              "frac": flops / (t_lsq * 1e-3) / p64, "flops": flops,
                                              "peak_source": "measured FP64 FMA probe (vof_probe_fma)"}},
                "nag": out["nag"], "lsq": out["lsq"]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the plain FP64 form (comparison)")
    ap.add_argument("--workload", default="deform3d")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--skip", type=int, default=0, help="untimed steps advanced before warm-up")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cases", type=int, default=256, help="batch workload: number of cases")
    ap.add_argument("--mlp", action="store_true", help="learned initial guess of the positioning (trained first)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default phase-flux launch (no autotuner)")
    ap.add_argument("--amr-every", type=int, default=8, help="octree_amr workload: steps between refinement cycles")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="batch workload: scale of the n ranges")
    ap.add_argument("--full-run", type=int, default=-1,
                    help="after the timed steps, run the whole case (t = 0 to its end) on the device and report the "
                         "L1 shape error against the initial field and the whole-case rate (1 on, 0 off; default: "
                         "on for the periodic deform3d and vortex_tet fields in the mixed form)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init(args)
    if args.workload == "batch":
        run_batch(args, world, rank, local)
        return
    if args.workload == "octree_amr":
        run_amr(args, world, rank, local)
        return
    if args.workload == "accuracy":
        run_accuracy(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1305_3417_gb300 import build, vof
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args)
    m = w.mesh
    prec = vof.MIXED if args.precision == "mixed" else vof.FP64
    ctx = vof.VofContext(m, precision=prec, device=local)
    learned = None
    if args.mlp and prec == vof.MIXED:
        learned = train_guess(local, args.workload)
        vof.vof_set_guess(ctx.h, learned["net"])
    total = args.skip + args.warmup + args.steps
    # per-step inputs resident in HBM before the timed region
    Fs = torch.from_numpy(w.F_spatial).to(dev)
    Us = torch.from_numpy(np.ascontiguousarray(w.U_spatial).reshape(-1)).to(dev)
    fac = []
    for k in range(total):
        t0 = k * w.dt
        tf = (w.field.tau_int(t0 + w.dt) - w.field.tau_int(t0)) / w.dt
        fac.append((tf, w.field.tau(t0 + 0.5 * w.dt)))
    Fk = [Fs * f for f, _ in fac]
    Uk = [Us * u for _, u in fac]
    alpha = torch.from_numpy(w.alpha0.copy()).to(dev)
    stats = torch.zeros(vof.S_LEN, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for k in range(args.skip + args.warmup):
        ctx.advect(alpha, Uk[k], Fk[k], w.dt, stats)
    torch.cuda.synchronize()
    # the phase-flux launch shape and staging chosen by the autotuner, on the
    # first timed step's state (it steps a copy)
    tuned = None
    if prec == vof.MIXED and not args.no_tune:
        k0 = args.skip + args.warmup
        cfg, tms = vof.vof_tune(ctx.h, alpha, Uk[k0], Fk[k0], w.dt)
        tuned = {"config": cfg, "stack": 92 if cfg // 256 == 0 else 56, "warps_per_block": (cfg // 16) % 16,
                 "grid_multiplier": cfg % 16, "step_ms": tms}
    a_start = alpha.clone()
    timed = [(Uk[args.skip + args.warmup + j], Fk[args.skip + args.warmup + j], w.dt) for j in range(args.steps)]
    st0 = ctx.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_stats = torch.zeros((args.steps, vof.S_LEN), dtype=torch.float64, device=dev)
    vof.vof_profile_begin(ctx.h, args.steps)
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        for j, (U, F, dt) in enumerate(timed):
            ctx.advect(alpha, U, F, dt, step_stats[j])
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    group_ms, nprof = vof.vof_profile_end(ctx.h)
    launches = vof.vof_last_launch_count(ctx.h) * args.steps
    st1 = ctx.status()
    ms_max = max_over_ranks(ms, world, dev)
    faces = world * args.steps * m.n_internal
    value = faces / (ms_max * 1e-3) / 1e6
    S = step_stats.cpu().numpy()
    drift = np.abs((S[:, 1] + S[:, 10] - S[:, 0]) / S[:, 0]).max()
    # the timed steps' algorithmic work, from the instrumented kernels on the same states
    work = counted_work(ctx, a_start, timed)
    peak32 = vof.vof_probe_fma(local, vof.MIXED)
    peak64 = vof.vof_probe_fma(local, vof.FP64)

    # ---- the other form on the same steps, for comparison (plain FP64 vs mixed)
    other = None
    if args.fp64_steps > 0 and world == 1:
        oprec = vof.FP64 if prec == vof.MIXED else vof.MIXED
        octx = vof.VofContext(m, precision=oprec, device=local)
        oa = torch.from_numpy(w.alpha0.copy()).to(dev)
        ost = torch.zeros(vof.S_LEN, dtype=torch.float64, device=dev)
        for k in range(args.skip + args.warmup):
            octx.advect(oa, Uk[k], Fk[k], w.dt, ost)
        torch.cuda.synchronize()
        ns = min(args.fp64_steps, args.steps)
        oa_start = oa.clone()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vof.vof_profile_begin(octx.h, ns)
        o0.record(stream)
        for j in range(ns):
            octx.advect(oa, *timed[j][:2], w.dt, ost)
        o1.record(stream)
        torch.cuda.synchronize()
        ogroup, onprof = vof.vof_profile_end(octx.h)
        oms = o0.elapsed_time(o1) / ns
        owork = counted_work(octx, oa_start, timed[:1])
        of32, of64, opf = work_flops(owork, oprec == vof.FP64)
        opk = peak64 if oprec == vof.FP64 else peak32
        ot_pf = ogroup["phase_flux"] / max(onprof, 1)
        other = {"precision": "fp64" if oprec == vof.FP64 else "mixed", "value": m.n_internal / (oms * 1e-3) / 1e6,
                 "unit": UNIT, "ms_per_step": oms, "steps": ns,
                 "group_ms_per_step": {g: v / max(onprof, 1) for g, v in ogroup.items()},
                 "roofline": {"kernel": "k_phase_flux" if oprec == vof.FP64 else "k_phase_flux_mixed", "bound": "alu",
                              "achieved": opf / (ot_pf * 1e-3) / 1e12, "peak": opk / 1e12, "unit": "TFLOP/s",
                              "frac": opf / (ot_pf * 1e-3) / opk,
                              "peak_source": f"measured {'FP64' if oprec == vof.FP64 else 'FP32'} FMA probe",
                              "work_per_launch": owork, "flops_per_launch": opf}}
        octx.close()
        del oa, ost, oa_start

    # ---- end to end through the C ABI with host buffers (copies in the timed region)
    ha = torch.from_numpy(w.alpha0.copy()).pin_memory()
    hstat = torch.zeros(vof.S_LEN, dtype=torch.float64).pin_memory()
    hF = [F.cpu().pin_memory() for _, F, _ in timed]
    hU = [U.cpu().pin_memory() for U, _, _ in timed]
    for k in range(args.skip + args.warmup):
        vof.vof_advect_host(ctx.h, ha, Uk[k].cpu(), Fk[k].cpu(), w.dt, hstat)
    torch.cuda.synchronize()
    barrier(world)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ej = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    th = []
    t_host0 = time.perf_counter()
    e2.record(stream)
    for j in range(args.steps):
        vof.vof_advect_host(ctx.h, ha, hU[j], hF[j], w.dt, hstat)
        ej[j].record(stream)
        th.append(time.perf_counter())
    e3.record(stream)
    t_host1 = time.perf_counter()
    torch.cuda.synchronize()
    host_calls = np.diff([t_host0] + th) * 1e3
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), world, dev)
    # per-call times (each call's events on the caller's stream)
    e2e_steps = [e2.elapsed_time(ej[0])] + [ej[j - 1].elapsed_time(ej[j]) for j in range(1, args.steps)]
    e2e = faces / (ms_e2e * 1e-3) / 1e6
    h2d = 8 * m.n_cells + 24 * m.n_cells + 8 * m.n_faces
    d2h = 8 * m.n_cells + 8 * vof.S_LEN
    link = host_link_gbps(stream, hU[0])
    diag = host_buffers_diag(stream, [ha] + hU + hF, dev)

    full = None
    do_full = args.full_run if args.full_run >= 0 else int(args.workload in ("deform3d", "vortex_tet")
                                                          and prec == vof.MIXED)
    if do_full and rank == 0:
        full = full_run_l1(ctx, w, dev)

    # ---- roofline of the dominant kernel group, and of the whole step
    pk, pk_src = peaks()
    per_launch = {g: v / max(nprof, 1) for g, v in group_ms.items()}
    dom = max(per_launch, key=per_launch.get)
    f32, f64, pf = work_flops(work, prec == vof.FP64)
    if dom == "phase_flux":
        alu = peak64 if prec == vof.FP64 else peak32
        achieved = pf / (per_launch[dom] * 1e-3) / 1e12
        traffic = captured_traffic(args.workload, m.shape[0], "fp64" if prec == vof.FP64 else "mixed") \
            if args.skip == 0 else None
        roof = {"kernel": "k_phase_flux" if prec == vof.FP64 else "k_phase_flux_mixed", "bound": "alu",
                "achieved": achieved, "peak": alu / 1e12, "unit": "TFLOP/s", "frac": achieved * 1e12 / alu,
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu capture)",
                "peak_source": f"measured {'FP64' if prec == vof.FP64 else 'FP32'} FMA probe (vof_probe_fma)",
                "work_per_launch": work, "flops_per_launch": pf}
    else:
        # HBM-bound groups: algorithmic bytes per internal face
        byts = BYTES_PER_FACE * m.n_internal
        achieved = byts / (per_launch[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": pk_src}
    roof["group_ms_per_step"] = per_launch
    # step: T_min = max(bytes / HBM, flops32 / peak32 + flops64 / peak64)
    byts = BYTES_PER_FACE * m.n_internal
    t_hbm = byts / (pk["hbm_gbs"] * 1e9) * 1e3
    t_alu = (f32 / peak32 + f64 / peak64) * 1e3
    t_min = max(t_hbm, t_alu)
    step_roof = {"bytes": byts, "flops32": f32, "flops64": f64, "t_hbm_ms": t_hbm, "t_alu_ms": t_alu,
                 "t_min_ms": t_min, "ms_per_step": ms_max / args.steps, "frac": t_min / (ms_max / args.steps),
                 "peak32_tflops": peak32 / 1e12, "peak64_tflops": peak64 / 1e12, "hbm_gbs": pk["hbm_gbs"],
                 "peak_source": f"FP32/FP64: measured FMA probe; HBM: {pk_src}"}
    band = float(S[:, 7].mean())

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, _ = cpu_baseline(w, steps=args.cpu_steps, one_thread=True)
    guess = None
    if learned is not None:
        it0, it1 = positioning_iterations(ctx, alpha, learned["net"])
        guess = {"iterations_per_cell_plain": it0, "iterations_per_cell_learned": it1,
                 "train_samples": learned["samples"], "train_loss": [learned["loss_first"], learned["loss_last"]],
                 "train_s": learned["train_s"]}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == vof.FP64 else "f32+f64",
                "data": "synthetic", "config": {**config(args, w), "tuned_launch": tuned},
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": ms_e2e / args.steps, "host_link_GBps": link, "host_buffers": diag,
                        "transfer": "alpha copied in and out, F copied (overlapping the previous step); pinned U "
                                    "read in place by the band kernels (the cells around band points): "
                                    "h2d_bytes_per_step counts all three arrays",
                        "call_ms": {"min": float(np.min(e2e_steps)), "median": float(np.median(e2e_steps)),
                                    "max": float(np.max(e2e_steps))},
                        "host_call_ms": {"min": float(host_calls.min()), "median": float(np.median(host_calls)),
                                         "max": float(host_calls.max()),
                                         "enqueue_total": (t_host1 - t_host0) * 1e3}},
                "gpu_launches": launches, "roofline": roof, "step_roofline": step_roof,
                "band_face_fluxes": {"value": world * band * args.steps / (ms_max * 1e-3) / 1e6, "unit": UNIT,
                                     "band_faces_per_step": band},
                "whole_case": None if full is None else {
                    "value": full["steps"] * m.n_internal / (full["gpu_ms"] * 1e-3) / 1e6, "unit": UNIT,
                    "ms_per_step": full["gpu_ms"] / full["steps"], "steps": full["steps"]},
                "cpu_baseline": base, "other_form": other,
                "learned_guess": guess,
                "clocks": clk.summary(),
                "quality": {"max_rel_volume_drift": float(drift), "alpha_min": float(S[:, 4].min()),
                            "alpha_max": float(S[:, 5].max()), "alpha_min_pre_bound": float(S[:, 2].min()),
                            "alpha_max_pre_bound": float(S[:, 3].max()),
                            "band_faces_per_step": band,
                            "interface_cells_per_step": float(S[:, 6].mean()),
                            "bound_sources_per_step": float(S[:, 12].mean()),
                            "bound_left_after_local": float(S[:, 13].mean()),
                            "bound_passes_max": float(S[:, 14].max()),
                            "bound_global_volume": float(S[:, 15].sum()),
                            "status_bits": int(st0 | st1), "full_run": full}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
