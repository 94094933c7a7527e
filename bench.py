"""Benchmark of the relativistic-beam EM PIC step on GB300.

Headline workload: the 3D beam in plasma -- grid 512 (z) x 256 (x) x 256 (y), dz = 0.02,
dx = dy = 0.05 c/omega_p, dt = 0.9 x the customised-stencil stability limit, moving window at c,
Gaussian electron beam (sigma_z = 0.5, sigma_r = 0.1, gamma = 2e4, 4e6 macro-particles) in a
uniform plasma of 2 particles per cell (67,108,864), quadratic shapes, customised M = 16 axial
stencil with the Sec. 3 current correction, FP32 fields and offsets; particles sorted by cell
every 20 steps.  One step = gather + Boris + Esirkepov deposition (fused) for both species,
current correction, field advance, window shift / injection when due.

Reported on one JSON line: particle-pushes/s of the whole step (value, the median of repeated
timed passes), cell-updates/s, the HBM roofline of the dominant kernel (the fused particle
kernel), an end-to-end number through the C ABI from pinned host buffers, the FP64 oracle
timed on the host cores on a stated sample (cpu_baseline), and under "secondary" the 2D beam in
plasma (2048 x 512), the field advance alone on grids far above L2 (2D 8192 x 2048 Yee and
M = 16, 3D 512 x 256 x 256 M = 16) with their HBM fractions, and the batched scan of 256
independent single-particle runs against one launch sequence per instance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torch.distributed.run, one independent replica per GPU (weak scaling,
no collective on the data path).
"""
import argparse
import json
import math
import os
import platform
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
REPEATS = 5                     # timed passes of --steps steps; the median is reported


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="headline only (profiling captures)")
    ap.add_argument("--small", action="store_true", help="reduced grid (profiling captures)")
    ap.add_argument("--fields-case", default=None, choices=["2d_yee", "2d_custom16", "3d_custom16", "2d_pair16"],
                    help="fields workload: run this grid only (profiling captures)")
    ap.add_argument("--sort-every", type=int, default=20, help="steps between particle sorts")
    ap.add_argument("--filter", action="store_true",
                    help="beam workloads with the 5-pass current filter along z (not the headline run)")
    ap.add_argument("--tile", type=int, default=None,
                    help="fields workload: force this field-advance tile variant instead of autotuning")
    ap.add_argument("--workload", default="beam3d", choices=["beam2d", "beam3d", "batch", "fields", "kspace"],
                    help="beam3d: the headline 3D 512 x 256 x 256 beam in plasma; beam2d: the 2D 2048 x 512 "
                         "beam in plasma; batch: 256 independent single-particle runs, batched launch vs "
                         "per-instance launches; fields: the field advance alone on grids above L2; kspace: "
                         "the k-space (spectral, [k1]_t) field advance alone")
    return ap.parse_args()


def workload(name, small=False, filt=False):
    """(grid, species, workload name) of a beam run (with the 5-pass current filter under filt)."""
    from paper_1910_13529_gb300 import workloads as wl
    if name == "beam3d":
        if small:
            (grid, sps), wname = wl.beam_plasma_3d(nz=256, nx=128, ny=128, n_beam=500_000), "beam_plasma_3d_small"
        else:
            (grid, sps), wname = wl.beam_plasma_3d(), "beam_plasma_3d_512x256x256"
    elif small:
        (grid, sps), wname = wl.beam_plasma(ndim=2, nz=512, nx=256, n_beam=250_000), "beam_plasma_2d_small"
    else:
        (grid, sps), wname = wl.beam_plasma(), "beam_plasma_2d_2048x512"
    if filt:
        grid["current_filter"] = True
        wname += "_filtered"
    return grid, sps, wname


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

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms",
                 str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)                       # first sample before the timed region
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


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------------- the FP64 oracle on the host ----

def host_cpu():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        ncores = len(os.sched_getaffinity(0))
    except Exception:
        ncores = os.cpu_count() or 1
    return model, ncores


def oracle_step_sample(grid, sps, n_full, z_slab, threads, steps=1, seed=0):
    """The FP64 oracle as it stands on a bounded piece of one step of the workload:
      particles -- gather, Boris, move and Esirkepov deposit of the sampled particles on the full
                   grid, scaled by n_full / n_sample;
      fields    -- the Sec. 3 correction and the field advance on a z slab of z_slab cells with the
                   full transverse grid, scaled by nz / z_slab (the cost is linear in the cells).
    Returns a dict with the estimated full-step time and its parts (seconds)."""
    from oracle import core as oc
    from oracle import fit
    from paper_1910_13529_gb300 import workloads as wl
    used = oc.set_threads(threads)
    nd = grid["ndim"]
    kappa = grid["dz"] / grid["dt"]
    C = fit.fit_coefficients(kappa)
    h = fit.correction_kernel(C, hlen=40)
    ny = grid.get("ny", 1)
    g = oc.Grid(nd, grid["nz"], grid["nx"], ny, grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C,
                shape=grid["shape"])
    gs = oc.Grid(nd, z_slab, grid["nx"], ny, grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C,
                 shape=grid["shape"])
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    Es, Bs, Js = gs.zeros(), gs.zeros(), gs.zeros()
    species = [oc.Species(wl.xi_of(sp, nd), sp["u"].T.astype(np.float64), sp["q"], sp["m"], sp["w"]) for sp in sps]
    n = sum(len(s.xi) for s in species)
    tp = tf = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        for s in species:
            eb = oc.gather(g, E, B, s.xi)
            oc.boris(eb, s.u, s.q * g.dt / (2.0 * s.m))
            xi1 = oc.move(g, s.xi, s.u)
            oc.deposit(g, s.xi, xi1, s.u, s.Q, J)
            s.xi = xi1
        t1 = time.perf_counter()
        oc.correct_j1(gs, h, Js)
        oc.field_advance(gs, Es, Bs, Js)
        t2 = time.perf_counter()
        tp += t1 - t0
        tf += t2 - t1
    tp /= steps
    tf /= steps
    oc.set_threads(1)
    t_part = tp * n_full / max(n, 1)
    t_field = tf * grid["nz"] / z_slab
    return dict(threads=used, n_sample=n, t_sample_s=tp + tf, t_particles_full_s=t_part, t_fields_full_s=t_field,
                t_step_full_s=t_part + t_field)


def cpu_baseline_3d(threads, frac, z_slab, steps=1, seed=0):
    from paper_1910_13529_gb300 import workloads as wl
    grid, sps, n_full = wl.beam_plasma_3d_sample(frac, seed=7 + seed)
    r = oracle_step_sample(grid, sps, n_full, z_slab, threads, steps=steps, seed=seed)
    cells = grid["nz"] * grid["nx"] * grid["ny"]
    r.update(n_full=n_full, cells=cells, pushes_per_s=n_full / r["t_step_full_s"],
             cell_updates_per_s=cells / r["t_fields_full_s"])
    return r, grid


def cpu_baseline_entry(r, grid, frac, z_slab, model, label):
    return {"value": r["pushes_per_s"], "unit": "particle-pushes/s", "cores": r["threads"], "kind": "oracle",
            "sample": f"{label}: one FP64 oracle step of the 512x256x256 beam in plasma on a sample -- "
                      f"particle phase on {r['n_sample']} particles ({100 * frac:.2f}% of {r['n_full']}), "
                      f"field phase (correction + field advance) on a {z_slab}x{grid['nx']}x{grid['ny']} z slab; "
                      f"{r['t_sample_s']:.1f} s measured, scaled to the full step by particle count and by "
                      f"cells",
            "ms_per_step_full_estimate": 1e3 * r["t_step_full_s"],
            "cell_updates_per_s": r["cell_updates_per_s"], "cpu_model": model}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores (all of them), on the headline configuration, each step a
    bounded sample of the 3D workload scaled to the full step."""
    if rank != 0:
        return
    model, ncores = host_cpu()
    frac, z_slab = 0.004, 64
    vals, ms = [], []
    r = grid = None
    for k in range(max(1, min(args.steps, 5))):
        r, grid = cpu_baseline_3d(ncores, frac, z_slab, seed=k)
        vals.append(r["pushes_per_s"])
        ms.append(1e3 * r["t_step_full_s"])
    value = float(np.median(vals))
    cpu = cpu_baseline_entry(r, grid, frac, z_slab, model, f"{len(vals)} sampled steps, median")
    cpu["value"] = value
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-pushes/s", "n_gpus": 0,
          "steps": len(vals), "warmup": 0, "ms_per_step": float(np.median(ms)),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic (seeded beam + quiet-start plasma, sampled)",
          "config": {"workload": "beam_plasma_3d_512x256x256", "grid": [512, 256, 256], "particles": r["n_full"]},
          "cpu_baseline": cpu,
          "e2e": {"value": value, "unit": "particle-pushes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------- ncu traffic of the dominant kernel ----

# ncu summaries committed under profiles/ that carry the DRAM traffic of a kernel class, with the
# SHA-1 of the source file the capture was built from
TRAFFIC_SOURCES = {
    ("particles", 2): ("profiles/push_deposit_2d_beam_plasma_2d.md", "paper_1910_13529_gb300/csrc/particle_kernels.cu"),
    ("particles", 3): ("profiles/push_deposit_3d_beam_plasma_3d_small.md", "paper_1910_13529_gb300/csrc/particle_kernels.cu"),
}


def captured_traffic(kind, ndim, units=None):
    """dram__bytes_read.sum + dram__bytes_write.sum of one step of the kernel class (all its
    launches in that step, the scope of roofline.achieved) from the committed ncu summary, or None
    when there is none or the kernel source has changed since the capture.  A summary taken on a
    reduced case states the particles of its captured step (units_per_step); the traffic is then
    scaled to `units` (particles per step of the timed run) in proportion."""
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
    m = re.search(r"traffic_bytes_per_step:\s*([0-9.eE+]+)", text)
    h = re.search(r"code_sha1:\s*([0-9a-f]{40})", text)
    if not m or not h or h.group(1) != digest:
        return None
    t = float(m.group(1))
    u = re.search(r"units_per_step:\s*([0-9.eE+]+)", text)
    if u and units:
        t *= units / float(u.group(1))
    return t


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


# ---------------------------------------------------------------- one beam-in-plasma run on the GPU ----

def build_sim(grid, sps, dev, sort_every):
    from paper_1910_13529_gb300.runtime import Simulation
    nd = grid["ndim"]
    n0 = [len(sp["iz"]) for sp in sps]
    cap_extra = 200_000 if nd == 2 else 4_000_000    # injection between two compacting sorts
    kw = {k: grid[k] for k in ("ndim", "nz", "nx", "ny", "dz", "dx", "dy", "dt", "shape", "solver",
                               "moving_window", "inject_species", "inject_ppc", "rho_bg")}
    kw["current_filter"] = grid.get("current_filter", False)
    sim = Simulation(device=str(dev), sort_every=sort_every, **kw)
    for s, sp in enumerate(sps):
        sim.add_species(s, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        cap=n0[s] + cap_extra)
    return sim, n0


def timed_passes(sim, steps, repeats, barrier, dev):
    """`repeats` passes of `steps` steps, each bracketed by a barrier and a synchronize, timed with
    CUDA events on the stream the library launches on (torch's current stream).  Returns the ms of
    each pass and the mean particle count over them."""
    import torch
    ms, counts = [], []
    d = sim.diag()
    counts.append(d["count"])
    for _ in range(repeats):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.step(steps)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        counts.append(sim.diag()["count"])
    return ms, float(np.mean(counts))


def kernel_breakdown(sim, steps):
    """Per-kernel-class times (CUDA events around every launch, on the launch stream) from a separate
    pass of the same length, so that the instrumentation stays out of the headline number."""
    from paper_1910_13529_gb300 import pic_timing, pic_timing_read
    c0 = sim.diag()["count"]
    pic_timing(sim.h, 1)
    sim.step(steps)
    kms, kl = pic_timing_read(sim.h, sim.stream)
    pic_timing(sim.h, 0)
    c1 = sim.diag()["count"]
    return kms, kl, 0.5 * (c0 + c1)


def interior_gauss_change(sim, G0, shifts0, margin):
    """max |G1 - G0| over interior nodes, G = d-.E - rho - rho_bg, in the lab frame: the residual
    of the initial state (the beam's charge without its field) is fixed in the lab frame, so G0
    is moved by the window shifts made since it was taken."""
    G1 = sim.gauss()
    s = int(sim.state()[1] - shifts0)
    nz = G1.shape[-1]
    d = G1[..., margin:nz - margin - s] - G0[..., margin + s:nz - margin]
    return float(d.abs().max().item())


def run_beam_secondary(args, dev, wname_sel):
    """The 2D beam in plasma (2048 x 512): pushes/s and the particle kernel's HBM fraction."""
    import torch
    grid, sps, wname = workload(wname_sel, filt=args.filter)
    sim, n0 = build_sim(grid, sps, dev, args.sort_every)
    tuned = sim.autotune()
    sim.step(args.warmup)
    torch.cuda.synchronize(dev)
    ms, count = timed_passes(sim, args.steps, 3, lambda: torch.cuda.synchronize(dev), dev)
    kms, kl, kcount = kernel_breakdown(sim, args.steps)
    peak, kind = measured_peak()
    med = float(np.median(ms))
    bpp = BYTES_PER_PUSH_2D if grid["ndim"] == 2 else BYTES_PER_PUSH_3D
    achieved = bpp * kcount * args.steps / (kms["particles"] / 1e3) / 1e9
    cells = grid["nz"] * grid["nx"] * grid.get("ny", 1)
    out = {"workload": wname, "particles": int(sum(n0)), "pushes_per_s": count * args.steps / (med / 1e3),
           "ms_per_step": med / args.steps, "cell_updates_per_s": cells * args.steps / (med / 1e3),
           "particle_kernel": {"achieved_GBps": achieved, "frac": achieved / peak, "peak_kind": kind,
                               "ms_per_step": kms["particles"] / args.steps,
                               "traffic": captured_traffic("particles", grid["ndim"], units=kcount)},
           "field_advance_GBps": BYTES_PER_CELL_UPDATE * cells * args.steps / (kms["fields"] / 1e3) / 1e9,
           "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
           "field_tile_variant": int(tuned[0]), "l2": "working set ~197 MB > 129 MB L2 (partly L2-resident)"}
    sim.close()
    return out


def kspace_cases(args):
    """The k-space field advance (Sec. 2.3 spectral solver, Sec. 3 [k]_1 = [k1]_t, Appendix B PSATD):
    2D 8192 x 2048 and 3D 512 x 256 x 256 at 0.9 of each solver's stability limit (PSATD: of one
    cell per step).  One advance = 9 forward and 6
    inverse FP32 transforms (cuFFT) and one update kernel over the modes; reported as
    cell-updates/s and as the finite-difference solver's 60 B/cell-update over its time."""
    import torch
    from paper_1910_13529_gb300 import (PIC_SOLVER_KT, PIC_SOLVER_PSATD, PIC_SOLVER_SPECTRAL, pic_cfl_dt_kspace,
                                        pic_timing, pic_timing_read)
    from paper_1910_13529_gb300.runtime import Simulation
    dev = torch.device("cuda:0")
    peak, kind = measured_peak()
    grids = [("2d_8192x2048", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dy=0.02)),
             ("3d_512x256x256", dict(ndim=3, nz=512, nx=256, ny=256, dz=0.02, dx=0.05, dy=0.05))]
    out = {}
    for gname, geo in grids:
        for sname, code in (("spectral", PIC_SOLVER_SPECTRAL), ("kt", PIC_SOLVER_KT), ("psatd", PIC_SOLVER_PSATD)):
            dt = 0.9 * pic_cfl_dt_kspace(geo["ndim"], code, geo["dz"], geo["dx"], geo["dy"])
            sim = Simulation(device="cuda:0", solver=sname, dt=dt, **geo)
            gen = torch.Generator(device="cuda:0").manual_seed(1)
            for t in (sim.E, sim.B, sim.J):
                t.copy_(torch.randn(t.shape, device="cuda:0", generator=gen) * 1e-3)
            sim.step(max(args.warmup, 3))
            torch.cuda.synchronize(dev)
            pic_timing(sim.h, 1)
            K = max(args.steps, 20)
            sim.step(K)
            kms, kl = pic_timing_read(sim.h, sim.stream)
            pic_timing(sim.h, 0)
            cells = sim.nz * sim.nx * sim.ny
            ms = float(kms["fields"]) / max(int(kl["fields"]), 1)
            gbs = BYTES_PER_CELL_UPDATE * cells / (ms / 1e3) / 1e9
            out[f"{gname}_{sname}"] = {"cell-updates/s": cells / (ms / 1e3), "ms_per_advance": ms,
                                       "achieved_GBps_at_60B": gbs, "frac": gbs / peak, "peak_kind": kind,
                                       "dt": dt}
            sim.close()
    return out


def fields_cases(args, which=None):
    """Field advance alone on grids far above L2: 2D 8192 x 2048 (Yee, customised M = 16 and the
    Sec. 3 split pair) and 3D 512 x 256 x 256 (customised), cell-updates/s and the HBM fraction at
    60 B/cell-update."""
    import torch
    from paper_1910_13529_gb300 import pic_fit_coefficients_b, pic_get_tuning, pic_set_tuning, pic_timing, pic_timing_read
    from paper_1910_13529_gb300 import workloads as wl
    from paper_1910_13529_gb300.runtime import Simulation
    dev = torch.device("cuda:0")
    peak, kind = measured_peak()
    cases = [("2d_8192x2048_yee", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dt=wl.DT_BEAM_2D, solver="yee")),
             ("2d_8192x2048_custom16", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dt=wl.DT_BEAM_2D,
                                            solver="custom", M=16)),
             ("3d_512x256x256_custom16", dict(ndim=3, nz=512, nx=256, ny=256, dz=0.02, dx=0.05, dy=0.05,
                                              dt=wl.DT_BEAM_3D, solver="custom", M=16)),
             # Sec. 3 split pair: Yee E side, B side fitted so that [k]_E1 [k]_B1 = [k1]_t^2
             ("2d_8192x2048_pair16", dict(ndim=2, nz=8192, nx=2048, dz=0.02, dx=0.02, dt=wl.DT_BEAM_2D,
                                          solver="custom", coef=[1.0],
                                          coef_b=pic_fit_coefficients_b(0.02 / wl.DT_BEAM_2D, [1.0], M=16)))]
    if which:
        cases = [c for c in cases if c[0] == which]
    out = {}
    for name, cfg in cases:
        sim = Simulation(device="cuda:0", **cfg)
        gen = torch.Generator(device="cuda:0").manual_seed(1)
        for t in (sim.E, sim.B, sim.J):
            t.copy_(torch.randn(t.shape, device="cuda:0", generator=gen) * 1e-3)
        if args.tile is None:
            tuned = sim.autotune()
        else:
            pic_set_tuning(sim.h, args.tile)
            tuned = pic_get_tuning(sim.h)
        # pic_step without particles: J zeroed, (customised stencil) J1 corrected, field advance
        # ping-ponging between the two buffers; the fields timing class holds the kernel alone
        sim.step(args.warmup)
        torch.cuda.synchronize(dev)
        pic_timing(sim.h, 1)
        K = max(args.steps, 20)
        sim.step(K)
        kms, kl = pic_timing_read(sim.h, sim.stream)
        pic_timing(sim.h, 0)
        cells = sim.nz * sim.nx * sim.ny
        kern_ms = float(kms["fields"]) / max(int(kl["fields"]), 1)
        gbs = BYTES_PER_CELL_UPDATE * cells / (kern_ms / 1e3) / 1e9
        out[name] = {"cell-updates/s": cells / (kern_ms / 1e3), "kernel_ms": kern_ms, "achieved_GBps": gbs,
                     "frac": gbs / peak, "peak_kind": kind, "tile_variant": int(tuned[0]),
                     "variant_ms": [float(x) for x in tuned[1]],
                     "l2": f"{cells * 60 / 1e6:.0f} MB moved per update > 129 MB L2"}
        sim.close()
    return out, K


def batch_configs(n=256, seed=4000):
    """The 256 instances of the batched vacuum scan (workloads.batched_vacuum_scan); the customised
    instances fit their M = 16 coefficients in pic_create at their own kappa."""
    from paper_1910_13529_gb300 import workloads as wl
    out = []
    for grid, gamma in wl.batched_vacuum_scan(n, seed):
        cfg = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver", "M")}
        out.append((cfg, gamma))
    return out


def batch_case(steps, warmup):
    """Batched scan of 256 instances against one pic_step call sequence per instance (the same
    kernels launched per instance), both timed with CUDA events on the same stream."""
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
    batch.step(warmup)
    for s1 in singles:
        s1.step(warmup)
    torch.cuda.synchronize(dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with ClockSampler(0) as clk:
        e0.record()
        batch.step(steps)
        e1.record()
        for s1 in singles:
            s1.step(steps)
        e2.record()
        torch.cuda.synchronize(dev)
    tb, ts = e0.elapsed_time(e1), e1.elapsed_time(e2)
    from paper_1910_13529_gb300 import pic_batch_get_tuning
    variants, vms = pic_batch_get_tuning(batch.b)
    for s1 in singles:
        s1.close()
    batch.close()
    return {"instances": len(cfgs), "cells_total": cells, "steps": steps,
            "custom_instances": sum(1 for c, _ in cfgs if c["solver"] == "custom"),
            "batched_cell_updates_per_s": cells * steps / (tb / 1e3),
            "per_instance_cell_updates_per_s": cells * steps / (ts / 1e3),
            "speedup_batched_over_per_instance": ts / tb, "ms_batched": tb, "ms_per_instance": ts,
            "field_variant_per_class": {"yee": variants[0], "custom16": variants[3]},
            "field_variant_ms": {"yee": list(map(float, vms[0])), "custom16": list(map(float, vms[3]))},
            "clocks": clk.summary()}


def tuning_case(iters=15):
    """The stencil-tuning run: 1024 x 256 vacuum, a rigid line of 64 electrons at gamma = 1e4,
    kappa = 4, loss = field energy behind the line after 500 steps, M = 4 coefficients from the
    Appendix C fit, adjoint with checkpoints every 50 steps; projected descent (tuning.py)."""
    import time as _t
    import torch
    from paper_1910_13529_gb300 import pic_fit_coefficients
    from paper_1910_13529_gb300 import workloads as wl
    from paper_1910_13529_gb300.runtime import StencilLoss
    from paper_1910_13529_gb300.tuning import tune_coefficients
    grid, sps = wl.rigid_line()
    C0 = pic_fit_coefficients(grid["dz"] / grid["dt"], M=4)
    problem = StencilLoss(grid, sps, nsteps=500, every=50)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    hist = tune_coefficients(problem, C0, iters=iters)
    torch.cuda.synchronize()
    dt = _t.perf_counter() - t0
    return {"grid": [1024, 256], "steps": 500, "checkpoint_every": 50, "C_appendix_c_fit": list(map(float, C0)),
            "C_tuned": list(map(float, hist["C_final"])), "loss": list(map(float, hist["loss"])),
            "loss_ratio": float(hist["loss"][-1] / hist["loss"][0]), "evaluations": hist["evals"],
            "s_per_loss_and_gradient": dt / hist["evals"]}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1910_13529_gb300 import encode_cells, pic_bind_species

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    grid, sps, wname = workload(args.workload, small=args.small, filt=args.filter)
    nd = grid["ndim"]
    bpp = BYTES_PER_PUSH_3D if nd == 3 else BYTES_PER_PUSH_2D
    sim, n0 = build_sim(grid, sps, dev, args.sort_every)
    tuned = sim.autotune()           # field-advance tile shape for this grid (timed, cached)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    sim.step(args.warmup)
    margin = (16 + 24 + 2) + (5 if grid.get("current_filter") else 0)
    G0 = sim.gauss()
    shifts0 = sim.state()[1]
    barrier()
    with ClockSampler(local_rank) as clk:
        ms_list, count = timed_passes(sim, args.steps, REPEATS, barrier, dev)
    barrier()
    ms = float(np.median(ms_list))
    dG = interior_gauss_change(sim, G0, shifts0, margin)
    rho_max = sim.diag()["rho_max"]
    del G0
    kms, klaunch, kcount = kernel_breakdown(sim, args.steps)
    barrier()
    ms_max, total_pushes, value = aggregate(ms, count, args.steps, world, dev)
    developed = None
    if world == 1 and not args.no_secondary and not args.small and args.workload == "beam3d":
        # the same run later, in the developed wake (step 400 of the configured 500)
        done = sim.state()[0]
        if done < 400:
            sim.step(400 - done)
        torch.cuda.synchronize(dev)
        ms_d, count_d = timed_passes(sim, args.steps, 3, barrier, dev)
        kms_d, _, kcount_d = kernel_breakdown(sim, args.steps)
        med_d = float(np.median(ms_d))
        ach_d = bpp * kcount_d * args.steps / (kms_d["particles"] / 1e3) / 1e9
        developed = {"steps_from": 400, "pushes_per_s": count_d * args.steps / (med_d / 1e3),
                     "ms_per_step": med_d / args.steps,
                     "kernel_ms_per_step": {k: v / args.steps for k, v in kms_d.items()},
                     "particle_kernel_frac": ach_d / measured_peak()[0]}
    cells = grid["nz"] * grid["nx"] * grid.get("ny", 1)
    cell_rate = cells * args.steps * world / (ms_max / 1e3)

    # roofline of the dominant kernel class
    dom = max(kms, key=kms.get)
    peak, peak_kind = measured_peak()
    if dom == "particles":
        algo = bpp * kcount * args.steps
        units_per_step = kcount
    else:
        algo = BYTES_PER_CELL_UPDATE * cells * args.steps
        units_per_step = cells
    achieved = algo / (kms[dom] / 1e3) / 1e9
    # DRAM bytes per launch of the class (ncu), scaled from a reduced capture by particles per step
    traffic = captured_traffic(dom, nd, units=kcount if dom == "particles" else None)

    # end to end through the C ABI from pinned host buffers: upload the initial state, run the
    # steps, download the final fields and particles
    host = []
    for s, sp in enumerate(sps):
        d = sim.species[s]
        host.append({k: torch.empty_like(d[k], device="cpu").pin_memory() for k in ("cell", "off", "u")})
        host[-1]["cell"].fill_(-1)
        n = n0[s]
        host[-1]["cell"][:n] = torch.from_numpy(encode_cells(sp["iz"], sp["ix"], sp["iy"], grid["nz"], grid["nx"]))
        host[-1]["off"][:, :n] = torch.from_numpy(sp["off"][: grid["ndim"]])
        host[-1]["u"][:, :n] = torch.from_numpy(sp["u"])
    hE = torch.zeros_like(sim.E, device="cpu").pin_memory()
    hB = torch.zeros_like(sim.B, device="cpu").pin_memory()
    out = [{k: torch.empty_like(v).pin_memory() for k, v in h.items()} for h in host]
    oE, oB = torch.empty_like(hE).pin_memory(), torch.empty_like(hB).pin_memory()
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
    sim.sort()                      # the uploaded particles come in generation order: sort them first
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
    e2e_value = sum(n0) * world * args.steps / (float(t.item()) / 1e3)
    working = (sum(sim.species[s]["cap"] for s in sim.species) * (bpp // 2) + cells * 4 * (6 + 6 + 3)) / 1e6
    sim.close()
    del host, out, hE, hB, oE, oB
    torch.cuda.empty_cache()

    secondary = {"cell-updates/s": cell_rate, "ms_per_pass": ms_list,
                 "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
                 "kernel_launches_per_step": {k: v / args.steps for k, v in klaunch.items()},
                 "gauss_change_interior_max": dG, "rho_max": rho_max}
    if developed:
        secondary["beam_plasma_3d_developed_wake"] = developed
    cpu = None
    if world == 1 and not args.no_secondary and args.workload == "beam3d" and not args.small:
        secondary["beam_plasma_2d"] = run_beam_secondary(args, dev, "beam2d")
        fc, kf = fields_cases(args)
        secondary["field_advance_large_grids"] = fc
        secondary["batched_scan"] = batch_case(max(args.steps, 20), max(args.warmup, 3))
        secondary["kspace_field_advance"] = kspace_cases(args)
        secondary["stencil_tuning"] = tuning_case()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nd == 3 and not args.small:
        model, ncores = host_cpu()
        r1, g1 = cpu_baseline_3d(1, 0.001, 16)
        rn, gn = cpu_baseline_3d(ncores, 0.004, 64)
        cpu = cpu_baseline_entry(rn, gn, 0.004, 64, model, f"all {rn['threads']} host threads")
        cpu["single_thread"] = cpu_baseline_entry(r1, g1, 0.001, 16, model, "1 thread")
        cpu["nproc"] = ncores
    if rank == 0:
        launches = int(sum(klaunch.values())) * REPEATS
        emit({"metric": METRIC, "value": value, "unit": "particle-pushes/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic (seeded beam + quiet-start plasma)",
              "config": {"workload": wname,
                         "grid": [grid["nz"], grid["nx"]] + ([grid["ny"]] if nd == 3 else []),
                         "particles": int(sum(n0)), "solver": "custom M=16 + Sec. 3 correction",
                         "shape": "quadratic", "moving_window": True, "sort_every": args.sort_every,
                         "current_filter": "5-pass" if grid.get("current_filter") else "none",
                         "timing": f"median of {REPEATS} passes of {args.steps} steps",
                         "l2": f"inputs larger than L2 (working set {working:.0f} MB > 129 MB)",
                         "parallelism": f"{world} independent replica(s)",
                         "field_tile_variant": int(tuned[0])},
              "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                           "algorithmic_bytes_per_unit": bpp if dom == "particles" else BYTES_PER_CELL_UPDATE,
                           "units_per_step": units_per_step,
                           "launches_per_step": klaunch[dom] / args.steps,
                           "kernel_ms_per_step": kms[dom] / args.steps,
                           "scope": "achieved and traffic: one step of the kernel class (all its launches)"},
              "cpu_baseline": cpu,
              "e2e": {"value": e2e_value, "unit": "particle-pushes/s", "h2d_bytes_per_step": h2d / args.steps,
                      "d2h_bytes_per_step": d2h / args.steps},
              "gpu_launches": launches,
              "clocks": clk.summary(),
              "secondary": secondary})


def run_batch(args):
    r = batch_case(args.steps, args.warmup)
    emit({"metric": METRIC, "value": r["batched_cell_updates_per_s"], "unit": "cell-updates/s", "n_gpus": 1,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_batched"] / args.steps,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
          "data": "synthetic (seeded instance parameters)",
          "config": {"workload": "batched_vacuum_scan", "instances": r["instances"], "cells_total": r["cells_total"],
                     "custom_instances": r["custom_instances"]},
          "secondary": r, "clocks": r["clocks"]})


def run_fields(args):
    tag = None
    if args.fields_case:
        tag = {"2d_yee": "2d_8192x2048_yee", "2d_custom16": "2d_8192x2048_custom16",
               "3d_custom16": "3d_512x256x256_custom16", "2d_pair16": "2d_8192x2048_pair16"}[args.fields_case]
    out, K = fields_cases(args, tag)
    best = out.get("2d_8192x2048_custom16", next(iter(out.values())))
    emit({"metric": METRIC, "value": best["cell-updates/s"], "unit": "cell-updates/s", "n_gpus": 1,
          "steps": K, "warmup": args.warmup, "ms_per_step": best["kernel_ms"], "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random fields)",
          "config": {"workload": "field_advance_large_grids", "l2": "inputs larger than L2"},
          "roofline": {"bound": "hbm", "kernel": "field_advance", "achieved": best["achieved_GBps"],
                       "peak": measured_peak()[0], "unit": "GB/s", "frac": best["frac"], "peak_kind": best["peak_kind"],
                       "traffic": None, "algorithmic_bytes_per_unit": 60},
          "cases": out})


def run_kspace(args):
    """The k-space field advance alone (spectral and [k1]_t solvers, 2D 8192 x 2048 and 3D
    512 x 256 x 256); the line's value is the 3D [k1]_t case."""
    out = kspace_cases(args)
    best = out["3d_512x256x256_kt"]
    emit({"metric": METRIC, "value": best["cell-updates/s"], "unit": "cell-updates/s", "n_gpus": 1,
          "steps": max(args.steps, 20), "warmup": max(args.warmup, 3), "ms_per_step": best["ms_per_advance"],
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
          "data": "synthetic (seeded random fields)",
          "config": {"workload": "kspace_field_advance", "l2": "inputs larger than L2"},
          "roofline": {"bound": "hbm", "kernel": "kspace_field_advance (cuFFT + update)",
                       "achieved": best["achieved_GBps_at_60B"], "peak": measured_peak()[0], "unit": "GB/s",
                       "frac": best["frac"], "peak_kind": best["peak_kind"], "traffic": None,
                       "algorithmic_bytes_per_unit": 60},
          "cases": out})


def main():
    args = parse()
    if args.workload == "kspace" and args.impl == "ours":
        run_kspace(args)
        return
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
