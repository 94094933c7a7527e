"""Benchmark of the relativistic-beam EM PIC step on GB300.

Workload: the 2D beam-in-plasma run -- grid 2048 (z) x 512 (x), dz = dx = 0.02 c/omega_p,
dt = 0.9 x the customised-stencil stability limit, moving window at c, bi-Gaussian electron
beam (sigma_z = 0.5, sigma_x = 0.2, gamma = 2e4 with 2% spread, 1e6 macro-particles) in a
uniform plasma of 4 particles per cell, quadratic shapes, customised M = 16 axial stencil,
FP32 fields and offsets; particles sorted by cell every 20 steps.  One step = gather + Boris
+ Esirkepov deposition (fused) for both species, current correction, field advance, window
shift / injection when due.

Reported: particle-pushes/s for the whole step (value), cell-updates/s, the HBM roofline of
the dominant kernel (the fused particle kernel), an end-to-end number through the C ABI from
pinned host buffers, and the FP64 oracle timed on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torch.distributed.run, one independent replica per GPU (weak scaling,
no collective on the data path).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_PUSH_2D = 48          # read + write cell (4) + offsets (2 x 4) + u (3 x 4)
BYTES_PER_PUSH_3D = 56          # read + write cell (4) + offsets (3 x 4) + u (3 x 4)
BYTES_PER_CELL_UPDATE = 60      # read E, B, J (9 x 4) + write E, B (6 x 4)
METRIC = "cell-updates/s and particle-pushes/s (% HBM roofline) at <=1e-5 rel err vs FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="reduced grid (profiling captures)")
    ap.add_argument("--fields-case", default=None, choices=["2d_yee", "2d_custom16", "3d_custom16"],
                    help="fields workload: run this grid only (profiling captures)")
    ap.add_argument("--sort-every", type=int, default=20, help="steps between particle sorts")
    ap.add_argument("--filter", action="store_true",
                    help="beam workloads with the 5-pass current filter along z (not the headline run)")
    ap.add_argument("--tile", type=int, default=None,
                    help="fields workload: force this field-advance tile variant instead of autotuning")
    ap.add_argument("--workload", default="beam2d", choices=["beam2d", "beam3d", "batch", "fields"],
                    help="beam2d: the bench workload; beam3d: the 3D 512 x 256 x 256 beam in plasma; "
                         "batch: 256 independent single-particle runs, batched launch vs per-instance "
                         "launches; fields: the field advance alone on grids above L2")
    return ap.parse_args()


def workload(args):
    """(grid, species, name) of the timed run (with the 5-pass current filter under --filter)."""
    (grid, sps), name = _workload(args)
    if getattr(args, "filter", False):
        grid["current_filter"] = True
        name += "_filtered"
    return (grid, sps), name


def _workload(args):
    from paper_1910_13529_gb300 import workloads as wl
    if args.workload == "beam3d":
        if args.small:
            return wl.beam_plasma_3d(nz=256, nx=128, ny=128, n_beam=500_000), "beam_plasma_3d_small"
        return wl.beam_plasma_3d(), "beam_plasma_3d"
    if args.small:
        return wl.beam_plasma(ndim=2, nz=512, nx=256, n_beam=250_000, behind_front=3.0), "beam_plasma_2d_small"
    return wl.beam_plasma(), "beam_plasma_2d"


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_baseline(grid, sps, frac=0.25, seed=0, steps=2):
    """FP64 oracle on the host: the full grid and a random fraction of the particles, `steps`
    steps; returns (particle pushes per second, seconds, particles)."""
    from oracle import core as oc
    from oracle import fit
    from paper_1910_13529_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    kappa = grid["dz"] / grid["dt"]
    C = fit.fit_coefficients(kappa)
    h = fit.correction_kernel(C, hlen=40)
    g = oc.Grid(grid["ndim"], grid["nz"], grid["nx"], grid.get("ny", 1), grid["dz"], grid["dx"], grid["dy"],
                grid["dt"], C=C, shape=grid["shape"])
    species, n = [], 0
    for sp in sps:
        sel = rng.random(len(sp["iz"])) < frac
        sub = {k: (v[..., sel] if isinstance(v, np.ndarray) and v.shape[-1] == len(sel) else v)
               for k, v in sp.items()}
        species.append(oc.Species(wl.xi_of(sub, grid["ndim"]), sub["u"].T.astype(np.float64), sp["q"], sp["m"],
                                  sp["w"]))
        n += int(sel.sum())
    sim = oc.Sim(g, species, h=h, moving_window=True, filt=grid.get("current_filter", False))
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step()
    dt = time.perf_counter() - t0
    return n * steps / dt, dt, n


def emit(obj):
    print(json.dumps(obj), flush=True)


# ncu summaries committed under profiles/ that carry the DRAM traffic of a kernel class, with the
# SHA-1 of the source file the capture was built from
TRAFFIC_SOURCES = {
    ("particles", 2): ("profiles/push_deposit_2d_beam_plasma_2d.md", "paper_1910_13529_gb300/csrc/particle_kernels.cu"),
    ("particles", 3): ("profiles/push_deposit_3d_beam_plasma_3d_small.md", "paper_1910_13529_gb300/csrc/particle_kernels.cu"),
}


def captured_traffic(kind, ndim):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed ncu summary, or
    None when there is none or the kernel source has changed since the capture."""
    import hashlib
    import re
    entry = TRAFFIC_SOURCES.get((kind, ndim))
    if entry is None:
        return None
    md, src = (os.path.join(ROOT, q) for q in entry)
    try:
        text = open(md).read()
        digest = code_sha1(open(src).read())
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"code_sha1:\s*([0-9a-f]{40})", text)
    if not m or not h or h.group(1) != digest:
        return None
    return float(m.group(1))


def code_sha1(source):
    """SHA-1 of a C++/CUDA source with its comments and white space removed: a capture stays
    valid across comment edits and is voided by any change to the code itself."""
    import hashlib
    import re
    code = re.sub(r"/\*.*?\*/", "", source, flags=re.S)
    code = re.sub(r"//[^\n]*", "", code)
    code = re.sub(r"\s+", "", code)
    return hashlib.sha1(code.encode()).hexdigest()


def aggregate(ms, pushes_per_step, steps, world, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's time and the work of all
    ranks (each rank runs its own replica, no collective on the data path).  Returns
    (max ms over ranks, total pushes over ranks, pushes/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, pushes_per_step * steps], dtype=torch.float64, device=device)
    if world > 1:
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        work = t[1:].clone()
        dist.all_reduce(work, op=dist.ReduceOp.SUM)
        ms_max, total = float(tmax.item()), float(work.item())
    else:
        ms_max, total = float(t[0].item()), float(t[1].item())
    return ms_max, total, total / (ms_max / 1e3)


def run_reference(args, rank, world):
    if rank != 0:
        return
    (grid, sps), wname = workload(args)
    n_total = sum(len(sp["iz"]) for sp in sps)
    vals, times = [], []
    # the oracle has nothing to warm up; at most three timed samples keep the run within minutes
    for k in range(max(1, min(args.steps, 3))):
        v, dt, n = oracle_baseline(grid, sps, frac=0.05, seed=k, steps=1)
        vals.append(v)
        times.append(dt)
    value = float(np.median(vals))
    sample = f"one FP64 oracle step on the full {grid['nz']}x{grid['nx']} grid with a 5% random sample " \
             f"({n} of {n_total}) of the particles, single thread"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-pushes/s", "n_gpus": 0,
          "steps": len(vals), "warmup": 0, "ms_per_step": 1e3 * float(np.median(times)),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": wname, "grid": [grid["nz"], grid["nx"]] + ([grid["ny"]] if grid["ndim"] == 3 else []),
                     "particles": n_total},
          "cpu_baseline": {"value": value, "unit": "particle-pushes/s", "cores": 1, "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": "particle-pushes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1910_13529_gb300 import pic_timing, pic_timing_read
    from paper_1910_13529_gb300.runtime import Simulation

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    (grid, sps), wname = workload(args)
    nd = grid["ndim"]
    bpp = BYTES_PER_PUSH_3D if nd == 3 else BYTES_PER_PUSH_2D
    n0 = [len(sp["iz"]) for sp in sps]
    cap_extra = 200_000 if nd == 2 else 4_000_000    # injection between two compacting sorts
    kw = {k: grid[k] for k in ("ndim", "nz", "nx", "ny", "dz", "dx", "dy", "dt", "shape", "solver",
                               "moving_window", "inject_species", "inject_ppc", "rho_bg")}
    kw["current_filter"] = grid.get("current_filter", False)
    sim = Simulation(device=str(dev), sort_every=args.sort_every, **kw)
    for s, sp in enumerate(sps):
        sim.add_species(s, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        cap=n0[s] + cap_extra)
    stream = sim.stream
    tuned = sim.autotune()           # field-advance tile shape for this grid (timed, cached)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    sim.step(args.warmup)
    d0 = sim.diag()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record()
        sim.step(args.steps)
        ev1.record()
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    d1 = sim.diag()
    # per-kernel-class times (CUDA events around every launch, on the launch stream) from a second
    # timed pass of the same length, so that the instrumentation stays out of the headline number
    pic_timing(sim.h, 1)
    sim.step(args.steps)
    kms, klaunch = pic_timing_read(sim.h, stream)
    pic_timing(sim.h, 0)
    d2 = sim.diag()
    barrier()
    pushes_per_step = 0.5 * (d0["count"] + d1["count"])
    ms_max, total_pushes, value = aggregate(ms, pushes_per_step, args.steps, world, dev)
    cells = grid["nz"] * grid["nx"] * grid.get("ny", 1)
    cell_rate = cells * args.steps * world / (ms_max / 1e3)

    # roofline of the dominant kernel class
    dom = max(kms, key=kms.get)
    peak, peak_kind = measured_peak()
    if dom == "particles":
        algo = bpp * 0.5 * (d1["count"] + d2["count"]) * args.steps
    else:
        algo = BYTES_PER_CELL_UPDATE * cells * args.steps
    achieved = algo / (kms[dom] / 1e3) / 1e9
    fa_gbs = BYTES_PER_CELL_UPDATE * cells * args.steps / (kms["fields"] / 1e3) / 1e9 if kms["fields"] else None

    # end to end through the C ABI from pinned host buffers: upload the initial state, run the
    # steps, download the final fields and particles
    host = []
    for s, sp in enumerate(sps):
        d = sim.species[s]
        host.append({k: torch.empty_like(d[k], device="cpu").pin_memory() for k in ("cell", "off", "u")})
        host[-1]["cell"].fill_(-1)
        from paper_1910_13529_gb300 import encode_cells
        n = n0[s]
        host[-1]["cell"][:n] = torch.from_numpy(encode_cells(sp["iz"], sp["ix"], sp["iy"], grid["nz"], grid["nx"]))
        host[-1]["off"][:, :n] = torch.from_numpy(sp["off"][: grid["ndim"]])
        host[-1]["u"][:, :n] = torch.from_numpy(sp["u"])
    hE = torch.zeros_like(sim.E, device="cpu").pin_memory()
    hB = torch.zeros_like(sim.B, device="cpu").pin_memory()
    out = [{k: torch.empty_like(v).pin_memory() for k, v in h.items()} for h in host]
    oE, oB = torch.empty_like(hE).pin_memory(), torch.empty_like(hB).pin_memory()
    from paper_1910_13529_gb300 import pic_bind_species
    h2d = sum(t.numel() * t.element_size() for h in host for t in h.values()) + 2 * hE.numel() * 4
    d2h = h2d
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.E.copy_(hE, non_blocking=True)
    sim.B.copy_(hB, non_blocking=True)
    for s in range(len(sps)):
        d = sim.species[s]
        for k in ("cell", "off", "u"):
            d[k].copy_(host[s][k], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        pic_bind_species(sim.h, s, d["cell"].data_ptr(), d["off"].data_ptr(), d["u"].data_ptr(), None, n0[s],
                         d["cap"], sps[s]["q"], sps[s]["m"], sps[s]["w"])
    sim.step(args.steps)
    oE.copy_(sim.E, non_blocking=True)
    oB.copy_(sim.B, non_blocking=True)
    for s in range(len(sps)):
        for k in ("cell", "off", "u"):
            out[s][k].copy_(sim.species[s][k], non_blocking=True)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_e2e = e0.elapsed_time(e1)
    t = torch.tensor([ms_e2e], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = total_pushes / (float(t.item()) / 1e3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nd == 2:
        v, dt, n = oracle_baseline(grid, sps, frac=0.5, steps=2)
        cpu = {"value": v, "unit": "particle-pushes/s", "cores": 1, "kind": "oracle",
               "sample": f"two FP64 oracle steps, full {grid['nz']}x{grid['nx']} grid, 50% random particle "
                         f"sample ({n} particles), {dt:.1f} s single-threaded"}
    if rank == 0:
        launches = int(sum(klaunch.values()))
        working = (sum(sim.species[s]["cap"] for s in sim.species) * (bpp // 2) + cells * 4 * (6 + 6 + 3)) / 1e6
        emit({"metric": METRIC, "value": value, "unit": "particle-pushes/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic (seeded beam + quiet-start plasma)",
              "config": {"workload": wname,
                         "grid": [grid["nz"], grid["nx"]] + ([grid["ny"]] if nd == 3 else []),
                         "particles": int(sum(n0)), "solver": "custom M=16",
                         "shape": "quadratic", "moving_window": True, "sort_every": args.sort_every,
                         "current_filter": "5-pass" if kw["current_filter"] else "none",
                         "l2": f"inputs larger than L2 (working set {working:.0f} MB > 129 MB)",
                         "parallelism": f"{world} independent replica(s)",
                         "field_tile_variant": int(tuned[0])},
              "secondary": {"cell-updates/s": cell_rate,
                            "field_advance_GBps": fa_gbs,
                            "kernel_ms": kms, "kernel_launches": klaunch},
              "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": captured_traffic(dom, nd),
                           "algorithmic_bytes_per_unit": bpp if dom == "particles" else BYTES_PER_CELL_UPDATE},
              "cpu_baseline": cpu,
              "e2e": {"value": e2e_value, "unit": "particle-pushes/s", "h2d_bytes_per_step": h2d / args.steps,
                      "d2h_bytes_per_step": d2h / args.steps},
              "gpu_launches": launches,
              "clocks": clk.summary(),
              "diag": {"count": d1["count"], "shifts": d1["shifts"], "gauss_max": d1["gauss_max"],
                       "rho_max": d1["rho_max"]}})
    sim.close()


KAPPA_CFL_CUSTOM_2D = 1.632488686516034   # customised-stencil stability fixed point, r = 1


def batch_configs(n=256, seed=4000):
    """256 independent 2D single-particle vacuum runs: nz ~ U{128..1024}, nx ~ U{64..256},
    log10 gamma ~ U[1, 5], dt = U[0.3, 0.99] x the instance's own solver limit, Yee or customised
    (M = 16 fitted at the instance's kappa) by a fair coin, dz = dx = 0.05, linear shape."""
    import math
    rng = np.random.default_rng(seed)
    d = 0.05
    out = []
    for i in range(n):
        nz = int(rng.integers(128, 1025))
        nx = int(rng.integers(64, 257))
        gamma = 10 ** rng.uniform(1, 5)
        frac = rng.uniform(0.3, 0.99)
        custom = bool(rng.integers(0, 2))
        dt = frac * (d / KAPPA_CFL_CUSTOM_2D if custom else d / math.sqrt(2))
        cfg = dict(ndim=2, nz=nz, nx=nx, dz=d, dx=d, dt=dt, shape=1, solver="custom" if custom else "yee", M=16)
        out.append((cfg, gamma))
    return out


def run_batch(args):
    import torch
    from paper_1910_13529_gb300 import workloads as wl
    from paper_1910_13529_gb300.runtime import Batch, Simulation
    dev = torch.device("cuda:0")
    cfgs = batch_configs()
    batch = Batch([c for c, _ in cfgs])
    singles = []
    cells = 0
    for i, (c, gamma) in enumerate(cfgs):
        _, sps = wl.single_particle(nz=c["nz"], nx=c["nx"], d=c["dz"], dt_over_dz=c["dt"] / c["dz"], gamma=gamma,
                                    z_cell=c["nz"] / 8, x_cell=c["nx"] / 2)
        sp = sps[0]
        batch.instances[i].add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"])
        s1 = Simulation(device="cuda:0", **c)
        s1.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"])
        singles.append(s1)
        cells += c["nz"] * c["nx"]
    K = args.steps
    batch.step(args.warmup)
    for s1 in singles:
        s1.step(args.warmup)
    torch.cuda.synchronize(dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with ClockSampler(0) as clk:
        e0.record()
        batch.step(K)
        e1.record()
        for s1 in singles:
            s1.step(K)
        e2.record()
        torch.cuda.synchronize(dev)
    tb, ts = e0.elapsed_time(e1), e1.elapsed_time(e2)
    value = cells * K / (tb / 1e3)
    emit({"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
          "ms_per_step": tb / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
          "data": "synthetic (seeded instance parameters)",
          "config": {"workload": "batched_vacuum_scan", "instances": len(cfgs), "cells_total": cells,
                     "custom_instances": sum(1 for c, _ in cfgs if c["solver"] == "custom")},
          "secondary": {"per_instance_launches_cell_updates_per_s": cells * K / (ts / 1e3),
                        "speedup_batched_over_per_instance": ts / tb, "ms_batched": tb, "ms_per_instance": ts},
          "clocks": clk.summary()})
    for s1 in singles:
        s1.close()
    batch.close()


def run_fields(args):
    """Field advance alone on grids far above L2: 2D 8192 x 2048 (Yee and customised M = 16) and
    3D 512 x 256 x 256 (customised), cell-updates/s and the HBM fraction at 60 B/cell-update."""
    import torch
    from paper_1910_13529_gb300 import pic_timing, pic_timing_read, workloads as wl
    from paper_1910_13529_gb300.runtime import Simulation
    dev = torch.device("cuda:0")
    peak, kind = measured_peak()
    cases = [("2d_8192x2048_yee", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dt=wl.DT_BEAM_2D, solver="yee")),
             ("2d_8192x2048_custom16", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dt=wl.DT_BEAM_2D,
                                            solver="custom", M=16)),
             ("3d_512x256x256_custom16", dict(ndim=3, nz=512, nx=256, ny=256, dz=0.02, dx=0.05, dy=0.05,
                                              dt=wl.DT_BEAM_3D, solver="custom", M=16))]
    if args.fields_case:
        tag = {"2d_yee": "2d_8192x2048_yee", "2d_custom16": "2d_8192x2048_custom16",
               "3d_custom16": "3d_512x256x256_custom16"}[args.fields_case]
        cases = [c for c in cases if c[0] == tag]
    out = {}
    for name, cfg in cases:
        sim = Simulation(device="cuda:0", **cfg)
        gen = torch.Generator(device="cuda:0").manual_seed(1)
        for t in (sim.E, sim.B, sim.J):
            t.copy_(torch.randn(t.shape, device="cuda:0", generator=gen) * 1e-3)
        if args.tile is None:
            tuned = sim.autotune()
        else:
            from paper_1910_13529_gb300 import pic_get_tuning, pic_set_tuning
            pic_set_tuning(sim.h, args.tile)
            tuned = pic_get_tuning(sim.h)
        # pic_step without particles: J zeroed, (customised stencil) J1 corrected, field advance
        # ping-ponging between the two buffers; the fields timing class holds the kernel alone
        sim.step(args.warmup)
        torch.cuda.synchronize(dev)
        pic_timing(sim.h, 1)
        K = max(args.steps // 10, 20)
        sim.step(K)
        kms, kl = pic_timing_read(sim.h, sim.stream)
        pic_timing(sim.h, 0)
        cells = sim.nz * sim.nx * sim.ny
        kern_ms = float(kms["fields"]) / max(int(kl["fields"]), 1)
        gbs = 60 * cells / (kern_ms / 1e3) / 1e9
        out[name] = {"cell-updates/s": cells / (kern_ms / 1e3), "kernel_ms": kern_ms, "achieved_GBps": gbs,
                     "frac": gbs / peak, "tile_variant": int(tuned[0]), "variant_ms": [float(x) for x in tuned[1]]}
        sim.close()
    best = out.get("2d_8192x2048_custom16", next(iter(out.values())))
    emit({"metric": METRIC, "value": best["cell-updates/s"], "unit": "cell-updates/s", "n_gpus": 1,
          "steps": K, "warmup": args.warmup, "ms_per_step": best["kernel_ms"], "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random fields)",
          "config": {"workload": "field_advance_large_grids", "l2": "inputs larger than L2"},
          "roofline": {"bound": "hbm", "kernel": "field_advance", "achieved": best["achieved_GBps"], "peak": peak,
                       "unit": "GB/s", "frac": best["frac"], "peak_kind": kind, "traffic": None,
                       "algorithmic_bytes_per_unit": 60},
          "cases": out})


def main():
    args = parse()
    if args.workload == "batch" and args.impl == "ours":
        run_batch(args)
        return
    if args.workload == "fields" and args.impl == "ours":
        run_fields(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
